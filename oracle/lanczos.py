"""Plain Lanczos (spectral bounds) and POLFED block Lanczos (oracle; test only).

lanczos_extrema: Sec. 2.1, Eq. lanczos_recurrence, with full
  reorthogonalisation (two classical Gram-Schmidt passes), stopping when the
  extreme Ritz pairs satisfy |b_{m+1} t_{mj}| <= tol * max|theta| (Eq. lan_criterion).

polfed: the workflow of Sec. 4.6 with the block Lanczos iteration of Sec. 2.2 and
  Sec. 4.3 applied to the filtered operator P(H~) (Clenshaw, Eq.
  clenshaw_chebyshev_prod):
    W_k = P V_k;  A_k = V_k^T W_k;  W_k -= sum_i V_i (V_i^T W_k)  (twice);
    W_k = V_{k+1} B_{k+1}  (QR, diag(B) >= 0);
    H_L gets A_k on the diagonal, B_{k+1} below and B_{k+1}^T above it.
  Convergence (Eq. blocklan_criterion): at checkpoints, diagonalise H_L and
  require ||B_{k+1} tau_kj|| <= tol for the nev_g largest Ritz values.
  Extraction (Sec. 4.3, last paragraph): u = V_{1:m} t, E = <u|H|u>,
  residual ||H u - E u||.  Readings where the paper is silent:
    * the converged block is rotated by a Rayleigh-Ritz with H on its span,
      so Ritz vectors of nearly equal filter values (the filter is almost
      symmetric about lambda) are separated by energy; E_i are then the
      Rayleigh quotients of the returned vectors;
    * the nev pairs returned are those nearest lambda (dense.nearest);
    * QR is column-wise Gram-Schmidt (two passes); a column whose remaining
      norm is below 1e-12 of the block norm is replaced by a fresh random
      vector orthogonal to everything so far, with a zero row in B.
  The start block is v[r, c] = uniform_pm_half(seed, r*s + c), orthonormalised.
"""
import math
import numpy as np

from pf_inputs import uniform_pm_half
from .chebyshev import rescale, filter_coefficients, clenshaw_apply
from .dos import guard_count, expected_krylov_dim
from .dense import nearest


def _cgs2(Vb, w):
    for _ in range(2):
        w = w - Vb @ (Vb.T @ w)
    return w


def lanczos_extrema(H, tol=1e-10, seed=12345, maxit=None, check_every=5):
    S = H.scipy()
    D = H.D
    maxit = min(D, 2000) if maxit is None else maxit
    v = uniform_pm_half(seed, np.arange(D))
    Vs = [v / np.linalg.norm(v)]
    al, be = [], []
    for i in range(maxit):
        w = S @ Vs[-1]
        a = float(Vs[-1] @ w)
        w = w - a * Vs[-1]
        if i > 0:
            w = w - be[-1] * Vs[-2]
        w = _cgs2(np.array(Vs).T, w)
        b = float(np.linalg.norm(w))
        al.append(a)
        be.append(b)
        m = len(al)
        if (m % check_every == 0) or m == maxit or m == D or b == 0.0:
            T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
            th, Y = np.linalg.eigh(T)
            r0, r1 = abs(b * Y[-1, 0]), abs(b * Y[-1, -1])
            hn = max(abs(th[0]), abs(th[-1]))
            if (r0 <= tol * hn and r1 <= tol * hn) or m == D or b == 0.0:
                return dict(emin=float(th[0]), emax=float(th[-1]), rmin=r0, rmax=r1, iters=m)
        Vs.append(w / b)
    raise RuntimeError("lanczos_extrema did not converge")


def padded_interval(emin, emax, rmin, rmax, pad=1e-3):
    """Rescaling interval [Emin - r - pad dE0, Emax + r + pad dE0], dE0 = (Emax - Emin)/2.

    Reading: Lanczos extremes lie inside the spectrum and |T_n(x)| grows
    exponentially for |x| > 1, so the interval of Eq. rescaledMatrix is widened.
    """
    de0 = 0.5 * (emax - emin)
    lo = emin - rmin - pad * de0
    hi = emax + rmax + pad * de0
    return 0.5 * (hi + lo), 0.5 * (hi - lo)


def start_block(D, s, seed):
    idx = np.arange(D * s, dtype=np.uint64)
    return uniform_pm_half(seed, idx).reshape(D, s)


def gs_qr(W, Vprev, seed, tag, rel_tol=1e-12):
    """Column-wise CGS2 QR with the breakdown rule described in the module docstring."""
    D, s = W.shape
    Q = np.zeros_like(W)
    R = np.zeros((s, s))
    wnorm = float(np.linalg.norm(W))
    for j in range(s):
        basis = Q[:, :j] if Vprev is None else np.hstack([Vprev, Q[:, :j]])
        w = W[:, j].copy()
        c = np.zeros(j)
        for _ in range(2):
            cj = Q[:, :j].T @ w
            w = w - Q[:, :j] @ cj
            c += cj
            if Vprev is not None:
                w = w - Vprev @ (Vprev.T @ w)
        R[:j, j] = c
        r = float(np.linalg.norm(w))
        if r <= rel_tol * max(wnorm, 1e-300):
            z = uniform_pm_half(seed ^ 0x5DEECE66D, np.arange(D, dtype=np.uint64) + np.uint64((tag * s + j) * D))
            z = _cgs2(basis, z)
            Q[:, j] = z / np.linalg.norm(z)
            R[j, j] = 0.0
        else:
            Q[:, j] = w / r
            R[j, j] = r
    return Q, R


def polfed(H, lam, nev, K, s, Ec, dE, tol=1e-10, seed=2024, eta=1.5, check_first=None,
           check_every=None, V1=None, return_state=False):
    """Eigenpairs of H nearest the absolute energy lam (Sec. 4.6 workflow, steps 4-6)."""
    D = H.D
    nev_g = min(guard_count(nev, D), D)
    Ht = rescale(H, Ec, dE)
    lam_t = (lam - Ec) / dE
    a = filter_coefficients(lam_t, K)
    Mmax = min(expected_krylov_dim(nev_g, s, eta), D)
    m_est = max(1, int(math.ceil(expected_krylov_dim(nev_g, s, 1.0) / s)))
    first = int(math.ceil(0.5 * m_est)) if check_first is None else check_first
    every = max(1, int(math.ceil(0.1 * m_est))) if check_every is None else check_every
    nblk = Mmax // s + 1
    V = np.zeros((nblk + 1, D, s))
    X = start_block(D, s, seed) if V1 is None else V1
    V[0], _ = gs_qr(X, None, seed, 0)
    HL = np.zeros(((nblk + 1) * s, (nblk + 1) * s))
    S = H.scipy()
    k = 0
    converged = False
    while True:
        W = clenshaw_apply(Ht, V[k], a)
        A = V[k].T @ W
        HL[k * s:(k + 1) * s, k * s:(k + 1) * s] = 0.5 * (A + A.T)
        Vb = V[:k + 1].transpose(1, 0, 2).reshape(D, (k + 1) * s)
        for _ in range(2):
            W = W - Vb @ (Vb.T @ W)
        Q, B = gs_qr(W, Vb, seed, k + 1)
        V[k + 1] = Q
        HL[(k + 1) * s:(k + 2) * s, k * s:(k + 1) * s] = B
        HL[k * s:(k + 1) * s, (k + 1) * s:(k + 2) * s] = B.T
        k += 1
        M = k * s
        last = (M + s > Mmax)
        if M >= nev_g and ((k >= first and (k - first) % every == 0) or last):
            th, T = np.linalg.eigh(HL[:M, :M])
            top = np.arange(M - nev_g, M)
            res = np.linalg.norm(B @ T[M - s:M, top], axis=0)
            if np.all(res <= tol):
                converged = True
                break
        if last:
            break
    Vm = V[:k].transpose(1, 0, 2).reshape(D, k * s)
    th, T = np.linalg.eigh(HL[:M, :M])
    top = np.arange(M - nev_g, M)
    U = Vm @ T[:, top]
    HU = S @ U
    G = U.T @ HU
    E, Z = np.linalg.eigh(0.5 * (G + G.T))
    U = U @ Z
    HU = HU @ Z
    res = np.linalg.norm(HU - U * E, axis=0)
    sel = nearest(E, lam, nev)
    out = dict(E=E[sel], U=U[:, sel], res=res[sel], theta=th[top], blocks=k, M=M,
               converged=converged, nev_g=nev_g, K=K)
    if return_state:
        out.update(V=Vm, HL=HL[:M, :M], B=B, T=T, Ht=Ht, a=a)
    return out
