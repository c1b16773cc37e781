"""GPU tests of serving (a12): continuous batching with admission by device footprint.

Bars: every request's result equals, bit for bit, the one-problem path on the same model
(basis, Hamiltonian, bounds, K, solve with the server's options) whatever else is resident;
the sum of resident footprints never exceeds the budget once two or more are resident;
memory returns to zero when the server drains; a failing request finishes with its own
status and leaves the others untouched.
"""
import numpy as np
import pytest

import pf_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


def _drain(sv, ids, max_steps=100000):
    out, peak_active, over_budget = {}, 0, False
    for _ in range(max_steps):
        q, a, f = sv.step()
        peak_active = max(peak_active, a)
        used, budget = sv.memory()
        if a >= 2 and used > budget:
            over_budget = True
        for i in ids:
            if i not in out:
                r = sv.take(i)
                if r is not None:
                    out[i] = r
        if len(out) == len(ids):
            break
    return out, peak_active, over_budget


def _standalone(pf, p, eps, nev, block, precision):
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    K = H.choose_K(eps, nev)
    return H.solve(eps, nev, K, block=block, precision=precision, return_vectors=False, raise_on_notconv=False)


def _requests():
    return [(pi.xxz_params(12, W=2.0, seed=1301), 0.5, 10), (pi.xxz_params(10, W=1.0, seed=1302), 0.4, 6),
            (pi.hubbard_params(5, 2, 3, U=1.0, W=3.0, seed=4301), 0.5, 8),
            (pi.xxz_params(12, W=5.0, seed=1303), 0.7, 12), (pi.qsun_params(N=3, L=6, seed=3301), 0.5, 10)]


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_server_results_equal_standalone(pf, precision):
    sv = pf.Server(block=8, precision=precision)
    reqs = _requests()
    ids = [sv.submit(pf.Model.from_params(p), eps, nev) for p, eps, nev in reqs]
    out, peak, _ = _drain(sv, ids)
    assert len(out) == len(ids)
    assert peak >= 2                          # the solves really were resident together
    for (p, eps, nev), i in zip(reqs, ids):
        r = out[i]
        ref = _standalone(pf, p, eps, nev, 8, precision)
        assert r.status == ref.status == 0
        assert np.array_equal(r.evals, ref.evals)
        assert np.array_equal(r.resid, ref.resid)
        assert r.report["blocks"] == ref.report["blocks"]
        assert r.latency_ms >= r.queue_ms >= 0.0
    assert sv.memory()[0] == 0
    sv.close()


def test_server_admission_budget(pf):
    reqs = [(pi.xxz_params(12, W=3.0, seed=1400 + r), 0.5, 10) for r in range(5)]
    D, L = 924, 12
    foot = pf.solve_footprint(D, D * (1 + L), 10, 8, "f32")
    sv = pf.Server(block=8, precision="f32", mem_budget_bytes=int(2.5 * foot))
    ids = [sv.submit(pf.Model.from_params(p), eps, nev) for p, eps, nev in reqs]
    out, peak, over = _drain(sv, ids)
    assert len(out) == 5 and not over
    assert peak == 2                          # 2.5 footprints admit exactly two at a time
    for (p, eps, nev), i in zip(reqs, ids):
        assert out[i].footprint_bytes == foot
        ref = _standalone(pf, p, eps, nev, 8, "f32")
        assert np.array_equal(out[i].evals, ref.evals)
    sv.close()


def test_server_max_active_and_oversize(pf):
    reqs = [(pi.xxz_params(10, W=1.0, seed=1500 + r), 0.5, 6) for r in range(4)]
    # a budget below one footprint: each request runs alone in an empty server
    sv = pf.Server(block=4, precision="f64", mem_budget_bytes=1024)
    ids = [sv.submit(pf.Model.from_params(p), eps, nev) for p, eps, nev in reqs]
    out, peak, _ = _drain(sv, ids)
    assert len(out) == 4 and peak == 1
    assert all(out[i].status == 0 for i in ids)
    sv.close()
    sv = pf.Server(block=4, precision="f64", max_active=3)
    ids = [sv.submit(pf.Model.from_params(p), eps, nev) for p, eps, nev in reqs]
    out, peak, _ = _drain(sv, ids)
    assert len(out) == 4 and peak == 3
    sv.close()


def test_server_failing_request_is_isolated(pf):
    sv = pf.Server(block=8, precision="f32")
    good = _requests()[:2]
    ids = [sv.submit(pf.Model.from_params(p), eps, nev) for p, eps, nev in good]
    # a quantum sun with N + L = 31 passes submission but its basis build refuses it
    bad = pi.qsun_params(N=3, L=28, seed=3399)
    bad_id = sv.submit(pf.Model.from_params(bad), 0.5, 4)
    out, _, _ = _drain(sv, ids + [bad_id])
    assert out[bad_id].status == 1            # PF_EINVAL from the basis build
    for (p, eps, nev), i in zip(good, ids):
        ref = _standalone(pf, p, eps, nev, 8, "f32")
        assert out[i].status == 0 and np.array_equal(out[i].evals, ref.evals)
    with pytest.raises(pf.PolfedError):
        sv.submit(pf.Model.from_params(good[1][0]), 0.5, 10 ** 6)   # nev > D
    with pytest.raises(pf.PolfedError):
        sv.submit(pf.Model.from_params(good[1][0]), 1.5, 4)         # eps outside [0, 1]
    sv.close()


@pytest.mark.parametrize("k", [19, 22])
def test_low_degree_many_pair_requests_converge(pf, k):
    """Requests of the serving stream (2 req/s, nev in {20, 50, 200}) with nev = 200 and K = 40-57:
    a reserve block joining after a pass that still gained 4-8x brought a spurious Ritz pair into
    the returned set; they must converge, and at L = 14 match dense diagonalisation."""
    from oracle import hamiltonian as oh, dense
    rq = pi.serving_stream(24, 2.0, Ls=(14, 16, 18), nevs=(20, 50, 200))[k]
    p = rq["params"]
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    K = H.choose_K(rq["eps"], rq["nev"])
    r = H.solve(rq["eps"], rq["nev"], K, block=16, precision="f32", return_vectors=False, raise_on_notconv=False)
    hn = r.report["hnorm"]
    assert r.status == 0 and np.max(r.resid) <= 1e-9 * hn
    if p.L == 14:
        w, _ = dense.eigh_dense(oh.build(p))
        lam = w[0] + rq["eps"] * (w[-1] - w[0])
        assert np.max(np.abs(r.evals - w[dense.nearest(w, lam, rq["nev"])])) <= 1e-10 * max(abs(w[0]), abs(w[-1]))
