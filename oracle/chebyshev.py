"""Rescaling, Chebyshev delta filter and Clenshaw recurrence (oracle; test only).

Eq. rescaledMatrix:  H~ = (H - E_c 1)/dE, E_c = (Emax+Emin)/2, dE = (Emax-Emin)/2.
Eq. transformation:  P(H~) = (1/chi) sum_{n=0..K} c_n T_n(H~), chi fixed by P(lam~)=1.
Eq. transformationCoefficients: c_n = sqrt(4 - 3 delta_{n0}) T_n(lam~),
                     T_n(lam~) = cos(n arccos lam~).
Eq. clenshaw_chebyshev_prod (Sec. 4.4), with a_n = c_n/chi:
    b_{K+1} = b_{K+2} = 0
    b_i = a_i V + 2 H~ b_{i+1} - b_{i+2},   i = K, ..., 1
    P(H~) V = a_0 V + H~ b_1 - b_2.
clenshaw_apply_cols: the same recurrence with coefficients of its own for each column of V.
"""
import numpy as np

from .hamiltonian import CSR


def rescale(H, Ec, dE):
    """H~ values: off-diagonal v/dE, diagonal (v - Ec)/dE (same structure)."""
    diag = H.diag_mask()
    data = np.where(diag, (H.data - Ec) / dE, H.data / dE)
    return CSR(D=H.D, indptr=H.indptr, indices=H.indices, data=data)


def chebyshev_T(n, x):
    """T_n(x) = cos(n arccos x) for |x| <= 1 (Eq. transformationCoefficients)."""
    return np.cos(np.asarray(n, dtype=np.float64) * np.arccos(x))


def filter_coefficients(lam_t, K):
    """a_n = c_n / chi, n = 0..K, with c_0 = T_0 = 1 and c_n = 2 T_n(lam~)."""
    n = np.arange(K + 1, dtype=np.float64)
    T = chebyshev_T(n, lam_t)
    c = np.where(n == 0, 1.0, 2.0) * T
    chi = np.sum(c * T)
    return c / chi


def filter_value(x, lam_t, K):
    """P_lam~^K(x) by the definition (direct sum), scalar or array x in [-1, 1]."""
    a = filter_coefficients(lam_t, K)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = np.arange(K + 1, dtype=np.float64)
    T = np.cos(np.outer(np.arccos(x), n))
    return T @ a


def clenshaw_step(Ht, V, B1, B2, a_i, alpha):
    """One step of the backward recurrence: a_i V + alpha (H~ B1) - B2.

    alpha = 2 for i >= 1 (b_i) and alpha = 1 for the closing line (P V).
    """
    return a_i * V + alpha * (Ht.scipy() @ B1) - B2


def clenshaw_apply(Ht, V, a):
    """W = P(H~) V by Eq. clenshaw_chebyshev_prod, in the paper's order."""
    K = len(a) - 1
    S = Ht.scipy()
    b1 = np.zeros_like(V)   # b_{i+1}
    b2 = np.zeros_like(V)   # b_{i+2}
    for i in range(K, 0, -1):
        b = a[i] * V + 2.0 * (S @ b1) - b2
        b2, b1 = b1, b
    return a[0] * V + (S @ b1) - b2


def clenshaw_apply_cols(Ht, V, C):
    """Column j of the result is P_j(H~) V[:, j], P_j the Chebyshev series with coefficients
    C[:, j] (C is (K+1) x s): clenshaw_apply run on each column with its own coefficients."""
    C = np.asarray(C, dtype=np.float64)
    out = np.empty_like(V)
    for j in range(V.shape[1]):
        out[:, [j]] = clenshaw_apply(Ht, V[:, [j]], C[:, j])
    return out


def forward_chebyshev_sum(Ht, V, a):
    """sum_n a_n T_n(H~) V by the forward three-term recurrence (Eq. chebyshev_definition).

    An independent evaluation of the same polynomial, used to pin clenshaw_apply.
    """
    S = Ht.scipy()
    t_prev = V.copy()
    out = a[0] * t_prev
    if len(a) == 1:
        return out
    t_cur = S @ V
    out = out + a[1] * t_cur
    for n in range(2, len(a)):
        t_next = 2.0 * (S @ t_cur) - t_prev
        out = out + a[n] * t_next
        t_prev, t_cur = t_cur, t_next
    return out
