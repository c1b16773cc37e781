"""GPU parity of the complex-Hermitian path (XXZ ring threaded by a flux phi per bond).

The device holds the real symmetric embedding [[A, -B], [B, A]] of H = A + iB; the oracle builds
H itself (complex128) and its embedding independently (oracle/hamiltonian.py).  Checks:
  * the embedded CSR (structure and values) bit for bit against the oracle's embedding;
  * pf_polfed_solve_complex against the oracle's dense complex diagonalisation: the nev
    eigenvalues nearest the target within 1e-10 ||H||, residuals ||H z - E z|| <= 1e-9 ||H||
    recomputed on the host with the oracle's complex H, eigenvectors equal up to a phase;
  * a real model is refused by the complex solve, and a complex model by the server.
"""
import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh, dense

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


@pytest.mark.parametrize("L,N,phi,bc", [(8, 4, 0.3, 0), (10, 5, 1.2, 0), (12, 6, -0.45, 0), (9, 4, 2.5, 1),
                                        (10, 3, 0.7, 0)])
def test_embedded_csr_bitexact(pf, L, N, phi, bc):
    p = pi.xxz_flux_params(L, phi, N=N, W=2.0, bc=bc, seed=7000 + L)
    Hg = pf.Hamiltonian.from_params(p)
    M = oh.real_embedding(oh.xxz_flux_hamiltonian(p))
    assert Hg.D == M.D and Hg.nnz == M.nnz
    rp, col, val = Hg.csr()
    assert np.array_equal(rp.cpu().numpy(), M.indptr)
    assert np.array_equal(col.cpu().numpy().astype(np.int64), M.indices)
    assert np.array_equal(val.cpu().numpy(), M.data)


@pytest.mark.parametrize("L,nev,s,eps,phi", [(10, 10, 4, 0.5, 0.37), (12, 20, 8, 0.5, 1.1), (12, 16, 8, 0.35, -0.8)])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_complex_solve_against_dense(pf, L, nev, s, eps, phi, precision):
    p = pi.xxz_flux_params(L, phi, W=2.0, seed=7100 + L)
    Hc = oh.xxz_flux_hamiltonian(p)
    A = Hc.dense()
    w, Z = np.linalg.eigh(A)
    hn = max(abs(w[0]), abs(w[-1]))
    lam = w[0] + eps * (w[-1] - w[0])
    sel = dense.nearest(w, lam, nev)
    Hg = pf.Hamiltonian.from_params(p)
    Hg.spectral_bounds()
    K = Hg.choose_K(eps, 2 * nev)
    r = Hg.solve_complex(eps, nev, K, block=s, precision=precision, target_abs=lam)
    assert r.status == 0
    assert np.max(np.abs(r.evals - w[sel])) <= 1e-10 * hn
    assert np.max(r.resid) <= 1e-9 * hn
    z = r.evecs.cpu().numpy()                              # (D, nev) complex
    assert z.shape == (Hc.D, nev)
    res_host = np.linalg.norm(A @ z - z * r.evals, axis=0)
    assert np.max(res_host) <= 1e-9 * hn
    assert np.abs(np.linalg.norm(z, axis=0) - 1.0).max() < 1e-12
    # eigenvectors of the oracle, up to a phase (the chosen levels are non-degenerate)
    ov = np.abs(np.einsum("ij,ij->j", Z[:, sel].conj(), z))
    assert np.min(ov) > 1.0 - 1e-8


def test_complex_solve_refuses_a_real_model_and_server_refuses_complex(pf):
    Hr = pf.Hamiltonian.from_params(pi.xxz_params(10, W=1.0, seed=1))
    Hr.spectral_bounds()
    with pytest.raises(pf.PolfedError):
        Hr.solve_complex(0.5, 4, 50, block=4)
    sv = pf.Server(block=4, precision="f32")
    with pytest.raises(pf.PolfedError):
        sv.submit(pf.Model.from_params(pi.xxz_flux_params(10, 0.4, W=1.0, seed=2)), 0.5, 4)
    sv.close()
