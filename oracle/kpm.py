"""Kernel polynomial method for the density of states (oracle; test infrastructure only).

Sec. 3.3, Eq. dos_kpm and App. B:
  rho(E~) = sum_k delta(E~ - E~_k), approximated by
  rho_KPM(x) = [mu_0 g_0 + 2 sum_{n=1}^{N-1} mu_n g_n T_n(x)] / (pi sqrt(1 - x^2)),
  mu_n = Tr T_n(H~), estimated stochastically as (1/R) sum_r <r| T_n(H~) |r> with R random
  vectors whose components are independent, zero mean and unit variance;
  g_n the Jackson kernel, g_n = [(N - n + 1) cos(pi n/(N+1)) + sin(pi n/(N+1)) cot(pi/(N+1))]/(N+1).
Eq. condition_for_K then fixes K with rho from KPM (dos.bisect_K after Eq. Nev).
Targets (Sec. 5.2): :maxdos is the E~ where rho_KPM is largest; (:offset, eta) moves from
there linearly to +1 (eta = 1) or -1 (eta = -1).

Readings: the random vectors are sqrt(12) (u - 1/2) with u the SplitMix64 uniforms of
pf_inputs (zero mean, unit variance), vector r is column r of a D x R block filled row-major
from one counter stream; :maxdos is searched on a uniform grid of 4001 points in
[-0.999, 0.999].
"""
import math
import numpy as np

import pf_inputs as pi
from . import dos


def random_block(D, R, seed):
    """D x R block, entry (i, r) = sqrt(12) (uniform01(seed, i R + r) - 1/2)."""
    return math.sqrt(12.0) * pi.uniform_pm_half(seed, np.arange(D * R)).reshape(D, R)


def moments(Ht, V, N):
    """mu_n = (1/R) sum_r v_r^T T_n(H~) v_r for n = 0..N-1, T_n by the three-term recurrence."""
    S = Ht.scipy()
    R = V.shape[1]
    mu = np.zeros(N)
    t_prev, t_cur = None, V.copy()
    for n in range(N):
        if n == 1:
            t_prev, t_cur = t_cur, S @ t_cur
        elif n >= 2:
            t_prev, t_cur = t_cur, 2.0 * (S @ t_cur) - t_prev
        mu[n] = float(np.sum(V * t_cur)) / R
    return mu


def jackson(N):
    n = np.arange(N, dtype=np.float64)
    a = math.pi / (N + 1)
    return ((N - n + 1) * np.cos(a * n) + np.sin(a * n) / math.tan(a)) / (N + 1)


def dos_kpm(x, mu):
    """rho_KPM at the points x (|x| < 1)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    N = len(mu)
    g = jackson(N)
    n = np.arange(N)
    T = np.cos(np.outer(np.arccos(x), n))
    coef = 2.0 * mu * g
    coef[0] = mu[0] * g[0]
    return (T @ coef) / (math.pi * np.sqrt(1.0 - x * x))


def maxdos(mu, npts=4001, edge=0.999):
    x = np.linspace(-edge, edge, npts)
    return float(x[int(np.argmax(dos_kpm(x, mu)))])


def offset_target(e_maxdos, eta):
    """(:offset, eta): e_maxdos + eta (1 - e_maxdos) for eta >= 0, e_maxdos + eta (e_maxdos + 1) below."""
    return e_maxdos + eta * (1.0 - e_maxdos) if eta >= 0 else e_maxdos + eta * (e_maxdos + 1.0)


def choose_K(lam_t, nev_g, mu):
    """K from Eq. condition_for_K with rho(lam~) from KPM (bisection in [K_approx/2, 2 K_approx])."""
    rho = float(dos_kpm(lam_t, mu)[0])
    return dos.bisect_K(lam_t, dos.window_halfwidth(nev_g, rho))
