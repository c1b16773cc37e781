"""Writes the stored eigenvalue sets that the large-sector parity tests compare with.

Only oracle/ (and the seeded inputs of pf_inputs) run here; nothing comes from the CUDA
path.  Each set is "the eigenvalues of H nearest the target lambda" of the workflow of
Sec. 4.6 (the target given as normalised energy eps: lambda = Emin + eps (Emax - Emin)),
listed by increasing |E - lambda| (ties: smaller E), more of them than the solve returns so
that a test can re-select the nearest ones around its own lambda.

Cases (python tests/golden/make_eigen_golden.py CASE [CASE ...]):
  xxz_L16_W3      XXZ L=16 periodic, J=1, Delta=1, W=3, seed 2001 (D = 12,870): dense
                  diagonalisation of the oracle's CSR (the plain definition), 140 values.
  xxz_L20_W1|W3|W5
                  XXZ L=20 periodic, J=1, Delta=1, W = 1, 3, 5 with seeds 2000, 2001, 2002
                  (D = 184,756): the three realisations of the L=20 benchmark.  Dense
                  diagonalisation would need 273 GB and a sparse LU of H - lambda for
                  shift-invert fills beyond this host's memory, so the oracle's own FP64
                  POLFED (Sec. 4.6 steps; scalar Lanczos s = 1, start seed 777, nev 110) runs
                  here; each value carries its residual ||H u - E u|| / ||H||.  The start
                  block and block width differ from the GPU solve's (seed 2024, s = 32), so
                  the two Krylov spaces are independent.
"""
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import pf_inputs as pi  # noqa: E402
from oracle import hamiltonian as oh, dense, dos as od, lanczos as ol, chebyshev as oc  # noqa: E402

EPS = 0.5
CASES = {
    "xxz_L16_W3": dict(L=16, W=3.0, seed=2001, method="dense", keep=140),
    "xxz_L20_W1": dict(L=20, W=1.0, seed=2000, method="polfed", keep=110),
    "xxz_L20_W3": dict(L=20, W=3.0, seed=2001, method="polfed", keep=110),
    "xxz_L20_W5": dict(L=20, W=5.0, seed=2002, method="polfed", keep=110),
}


def by_distance(E, lam):
    E = np.asarray(E)
    return np.lexsort((E, np.abs(E - lam)))


def run_dense(p, keep):
    H = oh.xxz_hamiltonian(p)
    w = np.linalg.eigvalsh(H.dense())
    emin, emax = float(w[0]), float(w[-1])
    lam = emin + EPS * (emax - emin)
    order = by_distance(w, lam)[:keep]
    return dict(emin=emin, emax=emax, lam=lam, hnorm=max(abs(emin), abs(emax)), E=w[order],
                r=np.zeros(keep), method="dense eigenvalues of the oracle CSR (numpy eigvalsh)")


def run_polfed(p, keep, s=1, seed=777):
    H = oh.xxz_hamiltonian(p)
    b = ol.lanczos_extrema(H, tol=1e-12)
    emin, emax = b["emin"], b["emax"]
    hnorm = max(abs(emin), abs(emax))
    lam = emin + EPS * (emax - emin)
    Ec, dE = ol.padded_interval(emin, emax, b["rmin"], b["rmax"])
    Ht = oc.rescale(H, Ec, dE)
    mu, G = od.exact_moments(Ht)
    K = od.choose_K((lam - Ec) / dE, od.guard_count(keep, H.D), H.D, mu, G)
    out = ol.polfed(H, lam, keep, K, s, Ec, dE, tol=1e-10, seed=seed)
    order = by_distance(out["E"], lam)
    return dict(emin=emin, emax=emax, lam=lam, hnorm=hnorm, E=out["E"][order], r=out["res"][order] / hnorm,
                method=(f"oracle FP64 POLFED (Sec. 4.6): s={s}, start seed {seed}, K={K}, nev={keep}, "
                        f"Krylov dim {out['M']}, converged={out['converged']}; extreme eigenvalues by the oracle's "
                        f"Lanczos to 1e-12 (residuals {b['rmin']:.1e}, {b['rmax']:.1e})"))


def write(name, c, res, seconds):
    path = os.path.join(HERE, f"{name}.txt")
    with open(path, "w") as f:
        f.write(f"# eigenvalues nearest the target (Sec. 4.6 workflow; target eps = {EPS}: "
                f"lambda = Emin + eps (Emax - Emin)), by increasing |E - lambda|\n")
        f.write(f"# model: XXZ (Eq. xxz) L={c['L']} N={c['L'] // 2} periodic J=1 Delta=1 W={c['W']} seed={c['seed']}\n")
        f.write(f"# method: {res['method']}\n")
        f.write(f"# written by tests/golden/make_eigen_golden.py {name} in {seconds:.0f} s\n")
        for k, key in (("emin", "emin"), ("emax", "emax"), ("lambda", "lam"), ("hnorm", "hnorm")):
            f.write(f"{k} {float(res[key])!r}\n")
        f.write("# E  residual/||H||\n")
        for e, r in zip(res["E"], res["r"]):
            f.write(f"{float(e)!r} {float(r):.3e}\n")
    print("wrote", path, flush=True)


def main(names):
    for name in names:
        c = CASES[name]
        p = pi.xxz_params(c["L"], W=c["W"], seed=c["seed"])
        t = time.time()
        res = run_dense(p, c["keep"]) if c["method"] == "dense" else run_polfed(p, c["keep"])
        write(name, c, res, time.time() - t)


if __name__ == "__main__":
    main(sys.argv[1:] or list(CASES))
