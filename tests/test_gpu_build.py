"""GPU parity: basis tables and CSR Hamiltonians vs the oracle, bit for bit (a1, a2)."""
import numpy as np
import pytest

import pf_inputs as pi
from oracle import basis as ob, hamiltonian as oh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


@pytest.mark.parametrize("L,N", [(2, 1), (6, 3), (12, 6), (13, 4), (20, 10)])
def test_xxz_basis_bitexact(pf, L, N):
    H = pf.Basis(pf.Model(kind=0, L=L, N=N))
    got = H.states().cpu().numpy()
    assert np.array_equal(got, ob.xxz_basis(L, N))


def test_hubbard_basis_tables(pf):
    b = pf.Basis(pf.Model(kind=2, L=12, N_up=6, N_dn=5))
    st = b.states().cpu().numpy()
    assert b.D == 924 * 792 and b.D_up == 924 and b.D_dn == 792
    assert np.array_equal(st[:924], ob.fixed_popcount_states(12, 6))
    assert np.array_equal(st[924:], ob.fixed_popcount_states(12, 5))


def _compare_csr(Hg, Ho):
    rp, col, val = (t.cpu().numpy() for t in Hg.csr())
    assert Hg.D == Ho.D and Hg.nnz == Ho.nnz
    assert np.array_equal(rp, Ho.indptr)
    assert np.array_equal(col.astype(np.int64), Ho.indices)
    # values: same operations in the same order on both sides -> identical bits
    assert np.array_equal(val, Ho.data), np.max(np.abs(val - Ho.data))


@pytest.mark.parametrize("L,W,bc,seed", [(2, 0.5, 0, 1), (3, 1.0, 0, 2), (12, 2.0, 0, 1001), (12, 2.0, 1, 1002),
                                         (16, 3.0, 0, 7)])
def test_xxz_csr_bitexact(pf, L, W, bc, seed):
    p = pi.xxz_params(L, N=L // 2, J=1.0, Delta=1.0, W=W, bc=bc, seed=seed)
    _compare_csr(pf.Hamiltonian.from_params(p), oh.xxz_hamiltonian(p))


def test_xxz_L20_csr_bitexact_and_count(pf):
    p = pi.xxz_params(20, W=1.0, seed=2000)
    Hg = pf.Hamiltonian.from_params(p)
    assert Hg.nnz == 2129556                  # 184756 diagonal + 1944800 off-diagonal (paper's n_nz)
    _compare_csr(Hg, oh.xxz_hamiltonian(p))


@pytest.mark.parametrize("N,L,seed", [(2, 4, 11), (3, 7, 3001), (3, 15, 3000)])
def test_qsun_csr_bitexact(pf, N, L, seed):
    p = pi.qsun_params(N=N, L=L, seed=seed)
    _compare_csr(pf.Hamiltonian.from_params(p), oh.qsun_hamiltonian(p))


@pytest.mark.parametrize("L,Nu,Nd,bc,seed", [(2, 1, 1, 1, 1), (6, 3, 3, 1, 4001), (7, 3, 2, 0, 5), (12, 6, 6, 1, 4000)])
def test_hubbard_csr_bitexact(pf, L, Nu, Nd, bc, seed):
    p = pi.hubbard_params(L, Nu, Nd, t=1.0, U=1.0, W=4.0, bc=bc, seed=seed)
    _compare_csr(pf.Hamiltonian.from_params(p), oh.hubbard_hamiltonian(p))


def test_rescaled_values_bitexact(pf):
    from oracle import chebyshev as oc
    p = pi.xxz_params(12, W=2.0, seed=1001)
    Hg = pf.Hamiltonian.from_params(p)
    Hg.set_rescale(-0.3, 7.25)
    Ec, dE, v64, v32 = Hg.rescaled()
    Ho = oc.rescale(oh.xxz_hamiltonian(p), -0.3, 7.25)
    assert (Ec, dE) == (-0.3, 7.25)
    assert np.array_equal(v64.cpu().numpy(), Ho.data)
    assert np.array_equal(v32.cpu().numpy(), Ho.data.astype(np.float32))


def test_start_block_matches_generator_definition(pf):
    V = pf.start_block(1000, 8, 2024).cpu().numpy()
    ref = pi.uniform_pm_half(2024, np.arange(8000)).reshape(1000, 8)
    assert np.array_equal(V, ref)
