"""GPU checks at the benchmark's full size (XXZ L=20, D=184756, nev=100, s=32, eps=0.5), in the
configuration bench.py times (FP32 filter, FP64 Lanczos, Rayleigh-Ritz and refinement).

The dense oracle cannot run here, so the checks use properties that hold at any size and
outputs the oracle can compute one by one:
  - residuals ||H u - E u|| recomputed on the CPU with the oracle's own CSR of H for a
    sample of returned pairs, <= 1e-9 ||H|| (the acceptance bar), and equal to the
    library's reported residuals to rounding;
  - Rayleigh quotients u^T H u (oracle CSR) equal to the returned eigenvalues;
  - orthonormality of the returned vectors;
  - the same eigenvalues (within 1e-10 ||H||) from an independent run of the plain FP64
    path with another start block (two runs that disagree on the set would differ here).
"""
import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


@pytest.fixture(scope="module")
def solved(pf):
    p = pi.xxz_params(20, W=1.0, seed=2000)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    K = H.choose_K(0.5, 100)
    r32 = H.solve(0.5, 100, K, block=32, precision="f32")
    r64 = H.solve(0.5, 100, K, block=32, precision="f64", seed=77, return_vectors=False)
    return p, H, K, r32, r64


def test_full_size_residuals_by_oracle(solved):
    p, H, K, r32, _ = solved
    Ho = oh.build(p).scipy()
    hn = r32.report["hnorm"]
    assert r32.status == 0 and np.max(r32.resid) <= 1e-9 * hn
    X = r32.evecs.cpu().numpy()                    # D x nev
    idx = np.linspace(0, 99, 12).astype(int)
    for j in idx:
        u = X[:, j]
        Hu = Ho @ u
        E = u @ Hu
        res = np.linalg.norm(Hu - r32.evals[j] * u)
        assert res <= 1e-9 * hn
        assert abs(res - r32.resid[j]) <= 1e-12 * hn
        assert abs(E - r32.evals[j]) <= 1e-12 * hn


def test_full_size_orthonormal(solved):
    _, _, _, r32, _ = solved
    X = r32.evecs
    G = (X.t() @ X).cpu().numpy()
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-10


def test_full_size_fp32_path_equals_fp64_path(solved):
    _, _, _, r32, r64 = solved
    hn = r32.report["hnorm"]
    assert r64.status == 0
    assert np.max(np.abs(np.sort(r32.evals) - np.sort(r64.evals))) <= 1e-10 * hn


def test_full_size_overlapped_batch_equals_alone(pf, solved):
    """Two full-size solves in one batch overlap on the device (the second's FP32 Lanczos phase
    beside the first's FP64 refinement, with both kernels capped in CTAs per SM); each result
    must equal the one-problem solve bit for bit."""
    p, H, K, r32, _ = solved
    p2 = pi.xxz_params(20, W=3.0, seed=2001)
    H2 = pf.Hamiltonian.from_params(p2)
    H2.spectral_bounds()
    K2 = H2.choose_K(0.5, 100)
    alone2 = H2.solve(0.5, 100, K2, block=32, precision="f32", return_vectors=False)
    res = pf.solve_batch([dict(H=H, eps=0.5, nev=100, K=K), dict(H=H2, eps=0.5, nev=100, K=K2)], block=32,
                         precision="f32", return_vectors=True)
    assert [r.status for r in res] == [0, 0]
    assert np.array_equal(res[0].evals, r32.evals) and np.array_equal(res[0].resid, r32.resid)
    assert torch.equal(res[0].evecs, r32.evecs)
    assert np.array_equal(res[1].evals, alone2.evals) and np.array_equal(res[1].resid, alone2.resid)
