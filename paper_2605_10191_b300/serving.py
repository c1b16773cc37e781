"""Request-stream driver for the continuous-batching server (pf_server_*).

A stream is a list of requests (model, eps, nev, arrival time in seconds).  The driver
submits each request once the host clock passes its arrival time, steps the server while
anything is queued or resident, and collects results as they finish.  Latency is measured
from arrival to completion: the time a request waits for the host loop to submit it (a step
in progress) plus the server's submit-to-completion time.
"""
import time
from dataclasses import dataclass

import numpy as np

from .api import Model, Server


@dataclass
class StreamResult:
    latencies_ms: np.ndarray      # per request, arrival -> completion
    queue_ms: np.ndarray          # per request, arrival -> admission
    statuses: np.ndarray
    eigenpairs: int               # returned pairs with residual within the tolerance
    makespan_s: float             # first arrival -> last completion
    steps: int
    peak_active: int
    results: list

    def summary(self):
        lat = self.latencies_ms
        return {"requests": int(len(lat)), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                "queue_p50_ms": float(np.percentile(self.queue_ms, 50)),
                "eigenpairs": int(self.eigenpairs), "makespan_s": self.makespan_s,
                "eigenpairs_per_s": self.eigenpairs / self.makespan_s if self.makespan_s > 0 else 0.0,
                "failed": int(np.sum(self.statuses != 0)), "steps": self.steps, "peak_active": self.peak_active}


def run_stream(server: Server, requests, res_tol=1e-9):
    """requests: dicts with keys params (a pf_inputs parameter record), eps, nev, t_arrival."""
    order = sorted(range(len(requests)), key=lambda k: requests[k]["t_arrival"])
    lag, sub_of = {}, {}
    out = [None] * len(requests)
    t0 = time.perf_counter()
    nxt, done, steps, peak = 0, 0, 0, 0
    t_last = 0.0
    while done < len(requests):
        now = time.perf_counter() - t0
        while nxt < len(order) and requests[order[nxt]]["t_arrival"] <= now:
            k = order[nxt]
            rq = requests[k]
            rid = server.submit(Model.from_params(rq["params"]), rq["eps"], rq["nev"])
            sub_of[rid] = k
            lag[rid] = (time.perf_counter() - t0) - rq["t_arrival"]
            nxt += 1
        q, a, f = server.step()
        steps += 1
        peak = max(peak, a)
        if f:
            for rid in list(sub_of):
                r = server.take(rid)
                if r is None:
                    continue
                k = sub_of.pop(rid)
                out[k] = (r, lag.pop(rid))
                done += 1
                t_last = time.perf_counter() - t0
        if q == 0 and a == 0 and nxt < len(order):
            wait = requests[order[nxt]]["t_arrival"] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
    lat = np.array([r.latency_ms + 1e3 * lg for r, lg in out])
    qms = np.array([r.queue_ms + 1e3 * lg for r, lg in out])
    st = np.array([r.status for r, _ in out])
    good = 0
    for r, _ in out:
        hn = r.report["hnorm"]
        if r.status == 0 or hn > 0:
            good += int(np.sum(r.resid <= res_tol * hn)) if hn > 0 else 0
    first = min(rq["t_arrival"] for rq in requests)
    return StreamResult(latencies_ms=lat, queue_ms=qms, statuses=st, eigenpairs=good, makespan_s=t_last - first,
                        steps=steps, peak_active=peak, results=[r for r, _ in out])


def run_one_at_a_time(requests, block=16, precision="f64", refine_precision="f64", res_tol=1e-9):
    """The same stream through a plain FIFO queue, one request at a time: each request starts when
    it has arrived and the previous one has finished (basis, CSR, bounds, K and the solve), and its
    latency is measured on the host clock from arrival to completion, as for the server."""
    import torch
    from .api import Hamiltonian
    order = sorted(range(len(requests)), key=lambda k: requests[k]["t_arrival"])
    lat = np.zeros(len(requests))
    st = np.zeros(len(requests), dtype=np.int64)
    good, service = 0, 0.0
    t0 = time.perf_counter()
    t_last = 0.0
    for k in order:
        rq = requests[k]
        wait = rq["t_arrival"] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ts = time.perf_counter()
        H = Hamiltonian.from_params(rq["params"])
        H.spectral_bounds()
        K = H.choose_K(rq["eps"], rq["nev"])
        r = H.solve(rq["eps"], rq["nev"], K, block=block, precision=precision, return_vectors=False,
                    raise_on_notconv=False, refine_precision=refine_precision)
        torch.cuda.synchronize()
        t_last = time.perf_counter() - t0
        service += time.perf_counter() - ts
        lat[k] = 1e3 * (t_last - rq["t_arrival"])
        st[k] = r.status
        hn = r.report["hnorm"]
        good += int(np.sum(r.resid <= res_tol * hn)) if hn > 0 else 0
        del H, r
    first = min(rq["t_arrival"] for rq in requests)
    span = t_last - first
    return {"requests": int(len(requests)), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "eigenpairs": int(good),
            "makespan_s": span, "eigenpairs_per_s": good / span if span > 0 else 0.0,
            "failed": int(np.sum(st != 0)), "service_s_total": service,
            "latency": "measured live: FIFO, one request at a time, host clock from arrival to completion"}
