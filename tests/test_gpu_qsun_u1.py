"""GPU parity of the U(1) quantum sun (Eq. qsun:U1): sector basis and CSR bit for bit against the
oracle (including the numerically normalised dot matrix), and solves against dense
diagonalisation (eigenvalues within 1e-10 ||H||, residuals <= 1e-9 ||H||)."""
import numpy as np
import pytest

import pf_inputs as pi
from oracle import hamiltonian as oh, dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


@pytest.mark.parametrize("N,L,M,seed", [(3, 6, 4, 1), (2, 8, 5, 2), (3, 9, 6, 3), (1, 5, 1, 4), (3, 13, 8, 5)])
def test_qsun_u1_csr_bitexact(pf, N, L, M, seed):
    p = pi.qsun_u1_params(N=N, L=L, M=M, seed=seed)
    Hg = pf.Hamiltonian.from_params(p)
    Ho = oh.build(p)
    rp, col, val = (t.cpu().numpy() for t in Hg.csr())
    assert Hg.D == Ho.D and Hg.nnz == Ho.nnz
    assert np.array_equal(rp, Ho.indptr)
    assert np.array_equal(col.astype(np.int64), Ho.indices)
    assert np.array_equal(val, Ho.data)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_qsun_u1_solve_matches_dense(pf, precision):
    p = pi.qsun_u1_params(N=3, L=8, M=5, seed=31)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    nev = 16
    K = H.choose_K(0.5, nev)
    w, _ = dense.eigh_dense(oh.build(p))
    hn = max(abs(w[0]), abs(w[-1]))
    lam = w[0] + 0.5 * (w[-1] - w[0])
    r = H.solve(0.5, nev, K, block=8, precision=precision, target_abs=lam)
    assert r.status == 0
    assert np.max(np.abs(r.evals - w[dense.nearest(w, lam, nev)])) <= 1e-10 * hn
    assert np.max(r.resid) <= 1e-9 * hn


def test_qsun_u1_kpm_degree_converges(pf):
    """A realisation whose Gaussian-DOS degree is too large (K = 3336: fewer than nev_g levels in the
    window, the refinement stalls) converges with the degree from the KPM density (K = 2098)."""
    p = pi.qsun_u1_params(N=3, L=15, M=9, seed=pi.config_seed(7, 2))
    H = pf.Hamiltonian.from_params(p)
    emin, emax, _, _ = H.spectral_bounds()
    Ec, dE = H.rescaled()[:2]
    mu = H.kpm_moments(N=512, R=32, seed=pi.config_seed(7, 2))
    K = pf.choose_K_kpm(mu, (emin + 0.5 * (emax - emin) - Ec) / dE, 50)
    assert K < H.choose_K(0.5, 50)
    r = H.solve(0.5, 50, K, block=16, precision="f32", return_vectors=False, raise_on_notconv=False)
    assert r.status == 0 and np.max(r.resid) <= 1e-9 * r.report["hnorm"]
