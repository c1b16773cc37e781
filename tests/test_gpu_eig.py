"""The H_L eigensolver (pf_sym_eig_select: tridiagonalisation, multisection, inverse iteration,
back-transformation) against dense LAPACK (numpy.linalg.eigh) on seeded symmetric matrices, at
orders that take each tridiagonalisation form: the thread-block-cluster kernel with the matrix in
distributed shared memory (n up to ~620), two launches per column (up to 3000) and four (above).

Bar: eigenvalues within 1e-12 ||A||; residuals ||A z - w z|| <= 1e-12 ||A||; unit eigenvectors
(1e-12), mutually orthogonal to 1e-9 (inverse iteration keeps vectors orthogonal by Gram-Schmidt only
within clusters closer than 1e-6 ||T||, beyond that each is accurate to ~eps ||T|| / gap); for
isolated eigenvalues the eigenvector equals LAPACK's up to sign.
Block-tridiagonal matrices shaped like H_L (s x s blocks, upper-triangular off-diagonal blocks)
and a matrix with an exactly repeated eigenvalue are included.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


def _dense(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return 0.5 * (M + M.T)


def _block_tridiagonal(nb, s, seed):
    rng = np.random.default_rng(seed)
    n = nb * s
    A = np.zeros((n, n))
    for k in range(nb):
        G = rng.standard_normal((s, s))
        A[k * s:(k + 1) * s, k * s:(k + 1) * s] = 0.5 * (G + G.T)
        if k + 1 < nb:
            B = np.triu(rng.standard_normal((s, s)))
            A[(k + 1) * s:(k + 2) * s, k * s:(k + 1) * s] = B
            A[k * s:(k + 1) * s, (k + 1) * s:(k + 2) * s] = B.T
    return A


def _check(pf, A, idx):
    n = A.shape[0]
    w, Z = pf.sym_eig_select(torch.from_numpy(A).cuda(), idx)
    ev, U = np.linalg.eigh(A)
    an = np.max(np.abs(ev))
    z = Z.cpu().numpy()
    assert z.shape == (n, len(idx))
    assert np.max(np.abs(w - ev[idx])) <= 1e-12 * an
    assert np.max(np.linalg.norm(A @ z - z * w, axis=0)) <= 1e-12 * an
    G = z.T @ z
    assert np.abs(np.diag(G) - 1.0).max() < 1e-12
    assert np.abs(G - np.eye(len(idx))).max() < 1e-9
    gaps = np.array([min(abs(ev[i] - ev[i - 1]) if i > 0 else np.inf, abs(ev[i + 1] - ev[i]) if i + 1 < n else np.inf)
                     for i in idx])
    iso = gaps > 1e-6 * an
    if iso.any():
        ov = np.abs(np.einsum("ij,ij->j", U[:, np.asarray(idx)[iso]], z[:, iso]))
        assert ov.min() > 1 - 1e-10


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 300, 448, 600, 700, 1350, 3010])
def test_dense_random_top_and_bottom(pf, n):
    A = _dense(n, 100 + n)
    q = min(n, 40)
    idx = list(range(n - q, n)) if n % 2 else list(range(q))
    _check(pf, A, idx)


@pytest.mark.parametrize("nb,s", [(12, 32), (20, 16), (30, 32), (50, 16)])
def test_block_tridiagonal_like_HL(pf, nb, s):
    A = _block_tridiagonal(nb, s, 7 * nb + s)
    n = nb * s
    _check(pf, A, list(range(n - min(n, 64), n)))


def test_scattered_indices_and_repeated_eigenvalue(pf):
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((90, 90)))
    ev = np.sort(rng.standard_normal(90))
    ev[40] = ev[41]                      # an exactly repeated eigenvalue
    A = (Q * ev) @ Q.T
    A = 0.5 * (A + A.T)
    _check(pf, A, [0, 5, 39, 40, 41, 42, 88, 89])


def test_invalid_arguments_are_refused(pf):
    A = torch.from_numpy(_dense(10, 1)).cuda()
    for idx in ([10], [-1], []):
        with pytest.raises((pf.PolfedError, ValueError)):
            pf.sym_eig_select(A, idx)
