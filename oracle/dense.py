"""Dense reference spectra (oracle; test infrastructure only).

  eigh_dense        LAPACK symmetric eigensolver via numpy (a library primitive)
  jacobi_eigh       cyclic Jacobi rotations in plain Python (independent check, tiny D)
  nearest           the nev eigenvalues nearest lambda: smaller |E - lambda| first,
                    then smaller E; returned ascending
  xx_spectrum       free-fermion closed form of the XX chain (Delta = 0, no field):
                    Jordan-Wigner gives H = (J/2) sum (c+_i c_{i+1} + h.c.) with the
                    boundary twist (-1)^(N-1), so one-particle energies J cos k with
                    k = 2 pi m / L (N odd) or 2 pi (m + 1/2) / L (N even)
  open_chain_levels free fermions on an open chain, -2 t cos(pi k/(L+1)), k = 1..L
"""
import itertools
import math
import numpy as np


def eigh_dense(H):
    return np.linalg.eigh(H.dense())


def jacobi_eigh(A, tol=1e-17, max_sweeps=60):
    """Cyclic-by-row Jacobi: returns (eigenvalues ascending, eigenvectors as columns).

    Sweeps until the off-diagonal Frobenius norm is below tol * ||A||_F.
    """
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    Q = np.eye(n)
    fro = math.sqrt(float(np.sum(A * A)))
    for _ in range(max_sweeps):
        off = math.sqrt(float(np.sum(np.triu(A, 1) ** 2)))
        if off <= tol * fro:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p], A[:, q] = c * ap - s * aq, s * ap + c * aq
                ap, aq = A[p, :].copy(), A[q, :].copy()
                A[p, :], A[q, :] = c * ap - s * aq, s * ap + c * aq
                qp, qq = Q[:, p].copy(), Q[:, q].copy()
                Q[:, p], Q[:, q] = c * qp - s * qq, s * qp + c * qq
    w = np.diag(A).copy()
    order = np.argsort(w)
    return w[order], Q[:, order]


def nearest(w, lam, nev):
    """Indices of the nev values nearest lam (ties: smaller value), sorted by value."""
    w = np.asarray(w)
    order = np.lexsort((w, np.abs(w - lam)))[:nev]
    return order[np.argsort(w[order], kind="stable")]


def _subset_sums(levels, N):
    return np.array(sorted(sum(c) for c in itertools.combinations(levels, N)))


def xx_spectrum(L, N, J=1.0):
    shift = 0.5 if N % 2 == 0 else 0.0
    ks = [2.0 * math.pi * (m + shift) / L for m in range(L)]
    return _subset_sums([J * math.cos(k) for k in ks], N)


def open_chain_levels(L, t=1.0):
    return [-2.0 * t * math.cos(math.pi * k / (L + 1)) for k in range(1, L + 1)]


def hubbard_free_spectrum(L, N_up, N_dn, t=1.0):
    eu = _subset_sums(open_chain_levels(L, t), N_up)
    ed = _subset_sums(open_chain_levels(L, t), N_dn)
    return np.sort((eu[:, None] + ed[None, :]).ravel())
