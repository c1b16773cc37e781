"""Pins of the oracle's filter, DOS/K rule and (block) Lanczos (CPU only)."""
import math
import os

import numpy as np
import pytest

import pf_inputs as pi
from oracle import hamiltonian as hm, dense, chebyshev as ch, dos, lanczos as lz

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _xxz12():
    H = hm.xxz_hamiltonian(pi.xxz_params(12, W=2.0, seed=1001))
    w, U = dense.eigh_dense(H)
    return H, w, U


@pytest.mark.parametrize("lam_t,K", [(0.0, 10), (0.3, 57), (-0.71, 200), (0.95, 33)])
def test_filter_is_one_at_target(lam_t, K):
    assert abs(ch.filter_value(lam_t, lam_t, K)[0] - 1.0) < 1e-12


def test_filter_coefficients_definition():
    a = ch.filter_coefficients(0.2, 7)
    T = np.cos(np.arange(8) * math.acos(0.2))
    c = np.array([1.0] + [2.0] * 7) * T
    assert np.allclose(a, c / np.sum(c * T), rtol=0, atol=1e-15)


def test_filter_against_closed_form_kernel():
    # sum_{n=0}^K c_n T_n(x) with c_0 = 1, c_n = 2 T_n(y) equals the Dirichlet-type sum
    # 1 + 2 sum cos(n t) cos(n p) = D_K(t - p) + D_K(t + p) - 1, D_K(u) = sin((K+1/2)u)/(2 sin(u/2)) * 2 / 2
    K, y = 41, 0.37
    p = math.acos(y)
    def dirich(u):
        return math.sin((K + 0.5) * u) / math.sin(u / 2.0) if abs(math.sin(u / 2)) > 1e-14 else 2 * K + 1.0
    chi = 0.5 * (dirich(0.0) + dirich(2 * p))
    for x in [-0.9, -0.2, 0.1, 0.36, 0.8]:
        t = math.acos(x)
        ref = 0.5 * (dirich(t - p) + dirich(t + p)) / chi
        assert abs(ch.filter_value(x, y, K)[0] - ref) < 1e-12


def test_window_edge_value_is_omega_reading():
    # Eq. K_approx with the sinc reading of Omega: P(lam~ +- delta) ~= 0.176 for large K
    for lam_t in (-0.6, 0.0, 0.3):
        K = 1000
        delta = dos.K_APPROX_CONSTANT * math.sqrt(1 - lam_t ** 2) / K
        v = ch.filter_value([lam_t - delta, lam_t + delta], lam_t, K)
        assert np.all(np.abs(v - dos.OMEGA) < 0.004)


def test_expected_krylov_dim_printed_formula():
    for l in open(os.path.join(GOLD, "expected_krylov_dim.txt")):
        if not l.startswith("#"):
            h, b, e, m = l.split()
            assert dos.expected_krylov_dim(int(h), int(b), float(e)) == int(m)


def test_clenshaw_equals_forward_sum_and_spectral_definition():
    H, w, U = _xxz12()
    Ec, dE = 0.5 * (w[-1] + w[0]), 0.5 * (w[-1] - w[0]) * 1.001
    Ht = ch.rescale(H, Ec, dE)
    V = lz.start_block(H.D, 4, 3)
    a = ch.filter_coefficients(0.13, 150)
    W1 = ch.clenshaw_apply(Ht, V, a)
    W2 = ch.forward_chebyshev_sum(Ht, V, a)
    Pdiag = ch.filter_value((w - Ec) / dE, 0.13, 150)
    W3 = U @ (Pdiag[:, None] * (U.T @ V))
    scale = np.abs(W3).max()
    assert np.abs(W1 - W3).max() < 1e-12 * max(scale, 1)
    assert np.abs(W2 - W3).max() < 1e-12 * max(scale, 1)


def test_clenshaw_step_composes_to_apply():
    H, w, _ = _xxz12()
    Ht = ch.rescale(H, 0.1, 7.0)
    V = lz.start_block(H.D, 3, 5)
    a = ch.filter_coefficients(-0.2, 9)
    b1 = np.zeros_like(V)
    b2 = np.zeros_like(V)
    for i in range(9, 0, -1):
        b2, b1 = b1, ch.clenshaw_step(Ht, V, b1, b2, a[i], 2.0)
    W = ch.clenshaw_step(Ht, V, b1, b2, a[0], 1.0)
    assert np.abs(W - ch.clenshaw_apply(Ht, V, a)).max() < 1e-14


def test_rescale_maps_spectrum():
    H, w, _ = _xxz12()
    Ec, dE = 0.3, 9.0
    wt = np.linalg.eigvalsh(ch.rescale(H, Ec, dE).dense())
    assert np.max(np.abs(wt - (w - Ec) / dE)) < 1e-14


def test_exact_moments_equal_spectrum_moments():
    H, w, _ = _xxz12()
    Ht = ch.rescale(H, -0.4, 8.0)
    mu, G = dos.exact_moments(Ht)
    wt = (w + 0.4) / 8.0
    assert abs(mu - wt.mean()) < 1e-14 and abs(G - wt.std()) < 1e-13


def test_K_bisection_agrees_with_K_approx():
    for lam_t in (-0.3, 0.0, 0.25):
        delta = 0.003
        kb = dos.bisect_K(lam_t, delta)
        ka = dos.k_approx(lam_t, delta)
        assert abs(kb - ka) / ka < 0.01


@pytest.mark.parametrize("n", [6, 12, 20])
def test_dense_eigh_against_jacobi(n):
    H = hm.xxz_hamiltonian(pi.xxz_params(6 if n == 20 else 4 + (n == 12) * 2, W=1.5, seed=n))
    A = H.dense()
    wj, Qj = dense.jacobi_eigh(A)
    w, _ = np.linalg.eigh(A)
    assert np.max(np.abs(w - wj)) < 1e-13 * np.abs(w).max()
    assert np.max(np.abs(A @ Qj - Qj * wj)) < 1e-12 * np.abs(w).max()


def test_lanczos_extrema_against_dense():
    H, w, _ = _xxz12()
    b = lz.lanczos_extrema(H, tol=1e-10)
    hn = max(abs(w[0]), abs(w[-1]))
    assert abs(b["emin"] - w[0]) <= 1e-10 * hn and abs(b["emax"] - w[-1]) <= 1e-10 * hn


def _solve_small(H, w, nev, s, eps, seed=2024, **kw):
    b = lz.lanczos_extrema(H)
    Ec, dE = lz.padded_interval(b["emin"], b["emax"], b["rmin"], b["rmax"])
    lam = b["emin"] + eps * (b["emax"] - b["emin"])
    Ht = ch.rescale(H, Ec, dE)
    mu, G = dos.exact_moments(Ht)
    nev_g = dos.guard_count(nev, H.D)
    K = dos.choose_K((lam - Ec) / dE, nev_g, H.D, mu, G)
    r = lz.polfed(H, lam, nev, K, s, Ec, dE, seed=seed, **kw)
    return r, lam


def test_polfed_oracle_matches_dense_xxz_L12():
    H, w, _ = _xxz12()
    r, lam = _solve_small(H, w, 20, 8, 0.5)
    sel = dense.nearest(w, lam, 20)
    hn = np.abs(w).max()
    assert r["converged"]
    assert np.max(np.abs(r["E"] - w[sel])) <= 1e-10 * hn
    assert np.max(r["res"]) <= 1e-9 * hn


@pytest.mark.parametrize("model", ["qsun", "hubbard"])
def test_polfed_oracle_matches_dense_other_models(model):
    if model == "qsun":
        H = hm.qsun_hamiltonian(pi.qsun_params(N=3, L=7, seed=3001))
    else:
        H = hm.hubbard_hamiltonian(pi.hubbard_params(6, 3, 3, t=1.0, U=1.0, W=4.0, seed=4001))
    w, _ = dense.eigh_dense(H)
    r, lam = _solve_small(H, w, 12, 4, 0.45)
    sel = dense.nearest(w, lam, 12)
    hn = np.abs(w).max()
    assert np.max(np.abs(r["E"] - w[sel])) <= 1e-10 * hn
    assert np.max(r["res"]) <= 1e-9 * hn


def test_block_lanczos_invariants():
    H, w, _ = _xxz12()
    b = lz.lanczos_extrema(H)
    Ec, dE = lz.padded_interval(b["emin"], b["emax"], b["rmin"], b["rmax"])
    r = lz.polfed(H, 0.0, 10, 120, 4, Ec, dE, check_first=6, check_every=1000, return_state=True)
    V, HL, Ht, a = r["V"], r["HL"], r["Ht"], r["a"]
    M = V.shape[1]
    assert np.abs(V.T @ V - np.eye(M)).max() < 1e-13
    PV = ch.clenshaw_apply(Ht, V, a)
    HLx = V.T @ PV
    # block tridiagonal projection, B upper triangular
    assert np.abs(HL - HLx).max() < 1e-12
    s = 4
    for k in range(M // s - 1):
        Bk = HL[(k + 1) * s:(k + 2) * s, k * s:(k + 1) * s]
        assert np.abs(np.tril(Bk, -1)).max() == 0.0
    # residual identity: ||P u - theta u|| = ||B_{m+1} tau_m|| (Sec. 2.2)
    th, T = np.linalg.eigh(HL)
    B = r["B"]
    for j in (M - 1, M - 3, M - 7):
        u = V @ T[:, j]
        lhs = np.linalg.norm(ch.clenshaw_apply(Ht, u[:, None], a)[:, 0] - th[j] * u)
        rhs = np.linalg.norm(B @ T[M - s:, j])
        assert abs(lhs - rhs) < 1e-12


# ---------------------------------------------------------------- KPM density of states
from oracle import kpm


def test_kpm_moments_with_basis_vectors_are_exact_traces():
    """With the D vectors sqrt(D) e_i the stochastic trace is the exact trace: mu_n = sum_k T_n(E~_k)."""
    H, w, _ = _xxz12()
    Ec, dE = -0.16, 6.72
    Ht = ch.rescale(H, Ec, dE)
    wt = (w - Ec) / dE
    N = 40
    mu = kpm.moments(Ht, math.sqrt(H.D) * np.eye(H.D), N)
    exact = np.array([np.sum(np.cos(n * np.arccos(wt))) for n in range(N)])
    assert np.max(np.abs(mu - exact)) < 1e-9 * H.D


def test_kpm_moments_equal_spectral_form():
    """Same random vectors: recurrence moments = (1/R) sum_r v^T U diag(T_n(E~)) U^T v."""
    H, w, U = _xxz12()
    Ec, dE = -0.16, 6.72
    Ht = ch.rescale(H, Ec, dE)
    V = kpm.random_block(H.D, 8, 77)
    mu = kpm.moments(Ht, V, 30)
    P = U.T @ V
    th = np.arccos((w - Ec) / dE)
    ref = np.array([np.sum(np.cos(n * th)[:, None] * P * P) / 8 for n in range(30)])
    assert np.max(np.abs(mu - ref)) < 1e-9 * H.D


def test_random_block_statistics():
    V = kpm.random_block(20000, 4, 5)
    assert abs(V.mean()) < 0.02 and abs(V.var() - 1.0) < 0.02


def test_jackson_kernel_values():
    g = kpm.jackson(64)
    assert abs(g[0] - 1.0) < 1e-14
    assert np.all(np.diff(g) < 0) and g[-1] > 0
    # N = 1: g_0 = [2 cos 0 + 0]/2 = 1
    assert abs(kpm.jackson(1)[0] - 1.0) < 1e-15


def test_kpm_dos_integrates_to_D_and_tracks_exact_density():
    H, w, _ = _xxz12()
    Ec, dE = -0.16, 6.72
    Ht = ch.rescale(H, Ec, dE)
    wt = (w - Ec) / dE
    mu = np.array([np.sum(np.cos(n * np.arccos(wt))) for n in range(60)])
    # integral over [-1, 1] with x = cos(t): int rho dx = mu_0 g_0 (the T_n, n >= 1, integrate to 0)
    t = (np.arange(20000) + 0.5) * math.pi / 20000
    integ = np.sum(kpm.dos_kpm(np.cos(t), mu) * np.sin(t)) * math.pi / 20000
    assert abs(integ - H.D) < 1e-6 * H.D
    # the smoothed density near the centre within 15 % of a histogram of the exact levels
    lo, hi = -0.05, 0.05
    count = np.sum((wt > lo) & (wt < hi))
    xs = np.linspace(lo, hi, 201)
    est = np.trapezoid(kpm.dos_kpm(xs, mu), xs)
    assert abs(est - count) < 0.15 * count


def test_kpm_maxdos_of_symmetric_spectrum_is_centre():
    # XX chain without fields: the spectrum is symmetric about 0 (particle-hole), so is rho_KPM
    H = hm.xxz_hamiltonian(pi.xxz_params(12, Delta=0.0, W=0.0, seed=1))
    w, _ = dense.eigh_dense(H)
    dE = 1.01 * max(abs(w[0]), abs(w[-1]))
    wt = w / dE
    mu = np.array([np.sum(np.cos(n * np.arccos(wt))) for n in range(40)])
    assert np.max(np.abs(mu[1::2])) < 1e-9 * H.D
    em = kpm.maxdos(mu)
    assert abs(em) < 1e-3
    assert kpm.offset_target(em, 0.0) == em
    assert abs(kpm.offset_target(0.2, 1.0) - 1.0) < 1e-15 and abs(kpm.offset_target(0.2, -1.0) + 1.0) < 1e-15
    assert abs(kpm.offset_target(0.2, 0.5) - 0.6) < 1e-15


def test_kpm_choose_K_satisfies_condition():
    H, w, _ = _xxz12()
    Ec, dE = -0.16, 6.72
    wt = (w - Ec) / dE
    mu = np.array([np.sum(np.cos(n * np.arccos(wt))) for n in range(80)])
    lam_t, nev_g = 0.05, 30
    K = kpm.choose_K(lam_t, nev_g, mu)
    delta = dos.window_halfwidth(nev_g, float(kpm.dos_kpm(lam_t, mu)[0]))
    edge = lambda k: float(np.max(ch.filter_value(np.array([lam_t - delta, lam_t + delta]), lam_t, k)))
    assert edge(K) <= dos.OMEGA < edge(K - 1)


# ---------------------------------------------------------------- Eq. dos_gaussian, Eq. Nev, K
@pytest.mark.parametrize("mu,G,D", [(0.0, 0.2, 924), (-0.13, 0.071, 184756)])
def test_gaussian_dos_normalisation_and_shape(mu, G, D):
    """Eq. dos_gaussian is a density of D states: its integral is D, its mean mu~, its variance
    G~^2, its peak D/(sqrt(2 pi) G~), and it falls to half the peak at mu~ +- G~ sqrt(2 ln 2).
    Quadrature (trapezoid on a fine grid over +-12 G~), not the formula, gives the moments."""
    x = np.linspace(mu - 12 * G, mu + 12 * G, 200001)
    rho = dos.gaussian_dos(x, D, mu, G)
    n0 = np.trapezoid(rho, x)
    m1 = np.trapezoid(x * rho, x) / n0
    m2 = np.trapezoid((x - m1) ** 2 * rho, x) / n0
    assert abs(n0 - D) <= 1e-9 * D
    assert abs(m1 - mu) <= 1e-9 * G
    assert abs(math.sqrt(m2) - G) <= 1e-8 * G
    assert abs(float(dos.gaussian_dos(mu, D, mu, G)) - D / (math.sqrt(2 * math.pi) * G)) <= 1e-12 * D / G
    half = float(dos.gaussian_dos(mu + G * math.sqrt(2 * math.log(2)), D, mu, G))
    assert abs(half / float(dos.gaussian_dos(mu, D, mu, G)) - 0.5) < 1e-12


def test_window_holds_about_nev_g_levels():
    """Eq. Nev with the Gaussian density of the exact moments: the window [lam~ - delta, lam~ + delta]
    of the K rule holds about nev_g eigenvalues of a many-body spectrum (disordered XXZ L=14,
    D = 3432, whose density is close to Gaussian); a lost factor 2 or sqrt(2 pi) in the density
    would put 0.5x, 2x or 2.5x as many there.  Counted on the dense spectrum."""
    H = hm.xxz_hamiltonian(pi.xxz_params(14, W=2.0, seed=1401))
    w = np.linalg.eigvalsh(H.dense())
    Ec, dE = 0.5 * (w[0] + w[-1]), 0.5 * (w[-1] - w[0]) * 1.001
    Ht = ch.rescale(H, Ec, dE)
    mu, G = dos.exact_moments(Ht)
    wt = (w - Ec) / dE
    for lam_t in (mu, mu + 0.5 * G, mu - 0.8 * G):
        for nev_g in (30, 150):
            delta = dos.window_halfwidth(nev_g, float(dos.gaussian_dos(lam_t, H.D, mu, G)))
            n = int(np.sum(np.abs(wt - lam_t) <= delta))
            assert 0.75 * nev_g <= n <= 1.3 * nev_g, (lam_t, nev_g, n)


def test_guard_rule_and_returned_edge_filter_value():
    """The guard reading: nev_g = ceil(g nev), g = 1.5 below D = 100,000 and 3 from there on.  With
    K from the window of nev_g levels, the nev-th level from the target sits at about
    (nev / nev_g) delta, where a sinc-shaped filter of that window (value Omega at delta, the
    reading of Eq. K_approx) is sinc(2.655 nev / nev_g): above 0.5 for either g, and above the
    magnitude of the sidelobe minimum (-0.217) by more than 2x."""
    assert dos.guard_count(10, 99999) == 15 and dos.guard_count(10, 100000) == 30
    assert dos.guard_count(7, 12870) == 11 and dos.guard_count(7, 184756) == 21
    x = np.linspace(4.0, 6.0, 20001)
    side = float(np.min(np.sin(x) / x))
    assert abs(side + 0.2172) < 1e-3
    for D in (50000, 200000):
        nev = 100
        t = 2.655 * nev / dos.guard_count(nev, D)
        edge = np.sin(t) / t
        assert edge > 0.5 and edge > 2 * abs(side)


def test_choose_K_is_K_approx_of_that_window():
    """choose_K = ceil(K_approx(lam~, delta)) with delta from Eq. Nev; the filter of that degree
    takes the value Omega at lam~ +- delta within the K_approx accuracy (Eq. condition_for_K)."""
    mu, G, D = 0.02, 0.15, 184756
    for lam_t, nev_g in ((0.0, 150), (0.3, 75), (-0.4, 300)):
        rho = float(dos.gaussian_dos(lam_t, D, mu, G))
        delta = nev_g / (2.0 * rho)
        K = dos.choose_K(lam_t, nev_g, D, mu, G)
        assert K == math.ceil(2.655 * math.sqrt(1 - lam_t ** 2) / delta)
        edge = ch.filter_value(np.array([lam_t - delta, lam_t + delta]), lam_t, K)
        # the filter is symmetric in theta = arccos x, not in x: at low degree (K = 159 here) the
        # two edges differ by ~0.01 to first order, their mean stays near Omega; a wrong
        # constant in Eq. K_approx (or a lost factor in delta) moves both by 0.1 or more
        assert abs(edge.mean() - dos.OMEGA) < 0.01 and np.all(np.abs(edge - dos.OMEGA) < 0.015)


# ---------------------------------------------------------------- QR breakdown branch
def _check_qr(W, Vprev, Q, R, deficient):
    D, s = W.shape
    assert np.abs(Q.T @ Q - np.eye(s)).max() < 1e-13                 # orthonormal, replacements too
    if Vprev is not None:
        assert np.abs(Vprev.T @ Q).max() < 1e-13                        # and orthogonal to the basis
    # W - Vprev (Vprev^T W) = Q R exactly up to rounding: the replaced columns' rows of R carry
    # no diagonal, the other entries reproduce W
    Wp = W if Vprev is None else W - Vprev @ (Vprev.T @ W)
    assert np.abs(Q @ R - Wp).max() < 1e-12 * max(1.0, np.abs(W).max())
    assert np.all(np.tril(R, -1) == 0.0) and np.all(np.diag(R) >= 0.0)
    for j in range(s):
        if j in deficient:
            assert R[j, j] == 0.0
        else:
            assert R[j, j] > 1e-6


def test_gs_qr_breakdown_branch():
    """gs_qr with rank-deficient blocks: a duplicated column, a zero column, and a column inside
    the span of the previous basis.  Each deficient column gets a fresh unit vector orthogonal to
    everything, with R[j, j] = 0; Q stays orthonormal and Q R reproduces the projected block."""
    D, s = 200, 6
    rng_cols = pi.uniform_pm_half(41, np.arange(D * s)).reshape(D, s)
    Vprev, _ = np.linalg.qr(pi.uniform_pm_half(42, np.arange(D * 3)).reshape(D, 3))
    W = rng_cols.copy()
    W[:, 2] = W[:, 0]                      # duplicate of column 0
    W[:, 4] = 0.0                          # zero column
    W[:, 5] = Vprev @ np.array([0.3, -1.2, 0.7])   # inside span(Vprev): zero after projection
    Q, R = lz.gs_qr(W, Vprev, seed=9, tag=1)
    _check_qr(W, Vprev, Q, R, deficient={2, 4, 5})
    # without a previous basis: two copies and a scaled copy
    W2 = rng_cols[:, :4].copy()
    W2[:, 1] = W2[:, 0]
    W2[:, 3] = -2.5 * W2[:, 0]
    Q2, R2 = lz.gs_qr(W2, None, seed=9, tag=0)
    _check_qr(W2, None, Q2, R2, deficient={1, 3})
    # the replacements are not a fixed vector: different tags (block steps) draw different ones
    Q3, _ = lz.gs_qr(W2, None, seed=9, tag=5)
    assert abs(float(Q3[:, 1] @ Q2[:, 1])) < 0.5


def test_polfed_through_breakdown_matches_dense():
    """A start block inside an invariant subspace (two exact eigenvectors far from the target):
    the first filtered block lies in the span of the start block, so every column breaks down
    and is replaced by fresh random vectors; the iteration then proceeds and still returns the
    nev eigenvalues nearest lambda."""
    H, w, U = _xxz12()
    b = lz.lanczos_extrema(H)
    Ec, dE = lz.padded_interval(b["emin"], b["emax"], b["rmin"], b["rmax"])
    lam = b["emin"] + 0.5 * (b["emax"] - b["emin"])
    Ht = ch.rescale(H, Ec, dE)
    mu, G = dos.exact_moments(Ht)
    nev = 10
    K = dos.choose_K((lam - Ec) / dE, dos.guard_count(nev, H.D), H.D, mu, G)
    V1 = U[:, [0, H.D - 1]].copy()        # the extreme eigenvectors: P V1 stays in their span
    r = lz.polfed(H, lam, nev, K, 2, Ec, dE, V1=V1, return_state=True)
    Vm = r["V"]
    assert np.abs(Vm.T @ Vm - np.eye(Vm.shape[1])).max() < 1e-12
    # the second block came from the breakdown: both of its B entries on the diagonal are zero
    B1 = r["HL"][2:4, 0:2]
    assert np.all(np.abs(np.diag(B1)) <= 1e-12)
    sel = dense.nearest(w, lam, nev)
    hn = np.abs(w).max()
    assert np.max(np.abs(r["E"] - w[sel])) <= 1e-10 * hn
    assert np.max(r["res"]) <= 1e-9 * hn


# ---------------------------------------------------------------- per-column coefficients
def test_clenshaw_apply_cols_columns_are_independent_filters():
    """clenshaw_apply_cols: column j equals the spectral definition U diag(P_j(E)) U^T v_j."""
    H, w, U = _xxz12()
    Ht = ch.rescale(H, -0.16, 6.72)
    wt = (w + 0.16) / 6.72
    s, K = 3, 40
    C = np.stack([ch.filter_coefficients(lt, K) for lt in (-0.3, 0.05, 0.6)], axis=1)
    V = pi.uniform_pm_half(5, np.arange(H.D * s)).reshape(H.D, s)
    got = ch.clenshaw_apply_cols(Ht, V, C)
    n = np.arange(K + 1)
    for j in range(s):
        Pj = np.cos(np.outer(np.arccos(wt), n)) @ C[:, j]
        ref = U @ (Pj * (U.T @ V[:, j]))
        assert np.abs(got[:, j] - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("K", [2, 3, 57, 400])
def test_residual_correction_form_of_the_filter(K):
    """The refinement's residual-correction form: for any theta, with beta_i the recurrence on the
    scalar theta (beta_i = a_i + 2 theta beta_{i+1} - beta_{i+2}), r = H~ u - theta u and
    d_i = 2 beta_{i+1} r + 2 H~ d_{i+1} - d_{i+2} (a per-column Clenshaw recurrence of degree K - 1
    with gamma_0 = beta_1, gamma_i = 2 beta_{i+1}),
        P(H~) u = P(theta) u + H~ d_1 - d_2 + beta_1 r,
    where the closing line H~ d_1 - d_2 + gamma_0 r is that recurrence's own.  Checked against the
    direct filter on near-eigenvectors (theta their Rayleigh quotients) and on random vectors."""
    H, w, U = _xxz12()
    Ec, dE = -0.16, 6.72
    Ht = ch.rescale(H, Ec, dE)
    a = ch.filter_coefficients(0.05, K)
    S = Ht.scipy()
    s = 4
    X = U[:, 400:400 + s] + 1e-4 * pi.uniform_pm_half(9, np.arange(H.D * s)).reshape(H.D, s)
    X /= np.linalg.norm(X, axis=0)
    for Y in (X, pi.uniform_pm_half(10, np.arange(H.D * s)).reshape(H.D, s)):
        theta = np.einsum("ij,ij->j", Y, S @ Y) / np.einsum("ij,ij->j", Y, Y)
        beta = np.zeros((K + 3, s))
        for i in range(K, 0, -1):
            beta[i] = a[i] + 2 * theta * beta[i + 1] - beta[i + 2]
        P_theta = a[0] + theta * beta[1] - beta[2]
        R = S @ Y - Y * theta
        G = np.empty((K, s))
        G[0] = beta[1]
        G[1:] = 2 * beta[2:K + 1]
        corr = Y * P_theta + ch.clenshaw_apply_cols(Ht, R, G)
        direct = ch.clenshaw_apply(Ht, Y, a)
        assert np.abs(corr - direct).max() < 1e-12 * max(1.0, np.abs(direct).max())
        # the correction itself is the size of the vectors' error, not of the vectors
        if Y is X:
            assert np.abs(corr - Y * P_theta).max() < 1e-2 * np.abs(direct).max()
