"""Density of states, filter width and polynomial degree (oracle; test only).

Eq. dos_gaussian: rho(E~) = D/(sqrt(2 pi) G~) exp(-(E~ - mu~)^2/(2 G~^2)), with
  mu~ and G~ the mean and standard deviation of the spectrum of H~, taken here
  exactly from traces: mu~ = Tr H~ / D, G~^2 = Tr H~^2 / D - mu~^2, and for a
  symmetric H~, Tr H~^2 = sum_ij (H~_ij)^2.
Eq. Nev: delta = N_ev / (2 rho(lam~)).
Eq. K_approx: K = 2.655 sqrt(1 - lam~^2) / delta.
Eq. condition_for_K: P_lam~^K(lam~ +- delta) = Omega, solved by bisection in
  [K_approx/2, 2 K_approx] (Sec. 4.2, last paragraph).
Omega is not given numerically in the paper ("slightly above the height of the
secondary peaks").  Reading used: for large K the filter is sinc-like in
theta = arccos x, and Eq. K_approx is the statement that the window edge sits at
(K + 1/2)|theta - phi| = 2.655, so Omega = sin(2.655)/2.655 ~= 0.1757.
Expected Krylov dimension (Sec. 5.5, printed as a one-line function):
  M_est = ceil((20.427 s + 1.696 nev) * eta).
"""
import math
import numpy as np

from .chebyshev import filter_value

K_APPROX_CONSTANT = 2.655
OMEGA = math.sin(K_APPROX_CONSTANT) / K_APPROX_CONSTANT


def exact_moments(Ht):
    """(mu~, G~) of the spectrum of H~ from traces of H~ and H~^2."""
    D = Ht.D
    tr = float(np.sum(Ht.data[Ht.diag_mask()]))
    tr2 = float(np.sum(Ht.data * Ht.data))
    mu = tr / D
    return mu, math.sqrt(max(tr2 / D - mu * mu, 0.0))


def gaussian_dos(E_t, D, mu_t, G_t):
    return D / (math.sqrt(2.0 * math.pi) * G_t) * np.exp(-(np.asarray(E_t) - mu_t) ** 2 / (2.0 * G_t * G_t))


def window_halfwidth(nev, rho):
    return nev / (2.0 * rho)


def k_approx(lam_t, delta):
    return K_APPROX_CONSTANT * math.sqrt(max(1.0 - lam_t * lam_t, 0.0)) / delta


def guard_count(nev, D):
    """nev_g = ceil(g nev), g = 3 for D >= 100,000 and 1.5 below: Ritz pairs converged (and
    eigenvalues put above the cutoff by K).  Where only KPM moments are known, D is mu_0.

    The paper does not fix the margin.  Reading: the nev pairs nearest lambda must have filter
    values well above the magnitude of the filter's negative sidelobe (the sinc minimum,
    ~ -0.217, under the reading of Eq. K_approx used for OMEGA), since that ratio bounds how
    fast a refinement pass removes errors there; at g = 1.5 the returned edge sits at
    P ~ sin(2.655/1.5)/(2.655/1.5) ~ 0.55, at g = 3 at ~ 0.87.  A larger guard lowers K
    (~ 1/nev_g) faster than it grows the Krylov space (~ 20.4 s + 1.7 nev_g, the printed fit of
    Sec. 5.5), which pays where the filter's products dominate (large D); where the Lanczos and
    Ritz work, growing with nev_g, dominates (small D), the smaller margin is kept.
    """
    g = 3.0 if D >= 100000 else 1.5
    return int(math.ceil(g * nev))


def choose_K(lam_t, nev_g, D, mu_t, G_t):
    rho = float(gaussian_dos(lam_t, D, mu_t, G_t))
    return max(1, int(math.ceil(k_approx(lam_t, window_halfwidth(nev_g, rho)))))


def bisect_K(lam_t, delta, omega=OMEGA):
    """Smallest K in [K_approx/2, 2 K_approx] with max P(lam~ +- delta) <= Omega (Eq. condition_for_K)."""
    k0 = k_approx(lam_t, delta)
    lo, hi = max(1, int(k0 // 2)), max(2, int(math.ceil(2 * k0)))

    def edge(K):
        x = np.clip([lam_t - delta, lam_t + delta], -1.0, 1.0)
        return float(np.max(filter_value(x, lam_t, K)))

    while hi - lo > 1:
        mid = (lo + hi) // 2
        if edge(mid) > omega:
            lo = mid
        else:
            hi = mid
    return hi


def expected_krylov_dim(nev, s, eta):
    return int(math.ceil((20.427 * s + 1.696 * nev) * eta))
