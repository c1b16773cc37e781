"""GPU parity of the J1-J2 and J1-J2-J3 chains (Eq. j1j2, Eq. j1j2j3): CSR bit for bit against
the oracle, and a solve against dense diagonalisation (eigenvalues within 1e-10 ||H||,
residuals <= 1e-9 ||H||)."""
import numpy as np
import pytest

import pf_inputs as pi
from oracle import hamiltonian as oh, dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


CASES = [
    dict(L=12, J2=0.5, J3=0.0, bc=0, seed=11),
    dict(L=12, J2=0.5, J3=0.225, bc=0, seed=12),
    dict(L=13, J2=0.5, J3=0.225, bc=1, seed=13),
    dict(L=10, J2=0.0, J3=0.3, bc=0, seed=14),      # range 3 without range 2
    dict(L=4, J2=0.7, J3=0.0, bc=0, seed=15),       # periodic L=4: each range-2 pair twice
    dict(L=16, J2=0.5, J3=0.225, bc=0, seed=16),
]


@pytest.mark.parametrize("c", CASES)
def test_j1j2j3_csr_bitexact(pf, c):
    p = pi.j1j2_params(c["L"], J2=c["J2"], J3=c["J3"], W=1.0, bc=c["bc"], seed=c["seed"])
    Hg = pf.Hamiltonian.from_params(p)
    Ho = oh.build(p)
    rp, col, val = (t.cpu().numpy() for t in Hg.csr())
    assert Hg.D == Ho.D and Hg.nnz == Ho.nnz
    assert np.array_equal(rp, Ho.indptr)
    assert np.array_equal(col.astype(np.int64), Ho.indices)
    assert np.array_equal(val, Ho.data)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_j1j2j3_solve_matches_dense(pf, precision):
    p = pi.j1j2_params(12, J2=0.5, J3=0.225, W=1.0, seed=21)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    nev = 20
    K = H.choose_K(0.5, nev)
    w, _ = dense.eigh_dense(oh.build(p))
    hn = max(abs(w[0]), abs(w[-1]))
    lam = w[0] + 0.5 * (w[-1] - w[0])
    r = H.solve(0.5, nev, K, block=8, precision=precision, target_abs=lam)
    assert r.status == 0
    assert np.max(np.abs(r.evals - w[dense.nearest(w, lam, nev)])) <= 1e-10 * hn
    assert np.max(r.resid) <= 1e-9 * hn
