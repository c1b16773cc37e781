"""CPU tests of the library's host-only entry points through the C ABI (no GPU is touched).

pf_kpm_dos, pf_kpm_target and pf_choose_K_kpm evaluate the kernel-polynomial density of states
(Sec. 3.3, App. B), the :maxdos / (:offset, eta) targets (Sec. 5.2) and the degree from
Eq. condition_for_K on moments the caller passes in; pf_solve_footprint is the server's admission
measure.  The moments here come from the oracle's stochastic trace on the CPU, so both sides see
the same array.  Bars: the density within 1e-10 D of the oracle's, the targets within 1e-12, K
equal as an integer (both sides bisect in FP64), the large-sector guard switching at the same D
on both sides, and the footprint covering the CSR and the Krylov basis of the printed size fit.
"""
import math

import numpy as np
import pytest

import pf_inputs as pi
from oracle import chebyshev as oc, dos as od, hamiltonian as oh, kpm, lanczos as ol


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


@pytest.fixture(scope="module")
def mu():
    """Moments of a disordered XXZ chain (L = 12, D = 924) from the oracle, N = 96, R = 16."""
    H = oh.build(pi.xxz_params(12, W=2.0, seed=1001))
    b = ol.lanczos_extrema(H, tol=1e-10)
    Ec, dE = ol.padded_interval(b["emin"], b["emax"], b["rmin"], b["rmax"])
    Ht = oc.rescale(H, Ec, dE)
    return kpm.moments(Ht, kpm.random_block(H.D, 16, 9), 96)


def test_kpm_dos_matches_oracle(pf, mu):
    x = np.linspace(-0.95, 0.95, 77)
    assert np.max(np.abs(pf.kpm_dos(mu, x) - kpm.dos_kpm(x, mu))) <= 1e-10 * mu[0]


def test_kpm_targets_match_oracle(pf, mu):
    em = kpm.maxdos(mu)
    assert abs(pf.kpm_target(mu, 0.0) - em) < 1e-12
    for eta in (-1.0, -0.6, 0.3, 1.0):
        assert abs(pf.kpm_target(mu, eta) - kpm.offset_target(em, eta)) < 1e-12


@pytest.mark.parametrize("scale", [1.0, 99999.0 / 924.0, 100000.0 / 924.0, 853776.0 / 924.0])
def test_choose_K_kpm_matches_oracle_on_both_sides_of_the_guard_switch(pf, mu, scale):
    """mu_0 stands for D in the guard rule: scaling the moments moves the density's normalisation
    across D = 100,000, where nev_g changes from ceil(1.5 nev) to ceil(3 nev), without moving its
    shape; the product's K must follow the oracle's rule on both sides of the switch."""
    m = mu * scale
    em = kpm.maxdos(m)
    for lam_t, nev in ((em, 20), (0.2, 10), (-0.4, 30), (0.55, 7)):
        K = pf.choose_K_kpm(m, lam_t, nev)
        assert K == kpm.choose_K(lam_t, od.guard_count(nev, m[0]), m), (scale, lam_t, nev)


def test_guard_switch_lowers_K(pf, mu):
    """At the same density shape, a larger guard widens the window of the K rule: K falls by about
    the ratio of the guards (1.5 / 3) across the switch."""
    lo, hi = mu * (99999.0 / mu[0]), mu * (100000.0 / mu[0])
    lam_t = kpm.maxdos(lo)
    K_lo, K_hi = pf.choose_K_kpm(lo, lam_t, 40), pf.choose_K_kpm(hi, lam_t, 40)
    assert 0.4 < K_hi / K_lo < 0.6


def test_kpm_host_errors(pf, mu):
    with pytest.raises(pf.PolfedError):
        pf.kpm_target(mu, 1.5)                     # eta outside [-1, 1]
    with pytest.raises(pf.PolfedError):
        pf.kpm_dos(mu, [1.0])                      # x on the edge of [-1, 1]
    with pytest.raises(pf.PolfedError):
        pf.choose_K_kpm(mu, 1.0, 10)               # target on the edge
    with pytest.raises(pf.PolfedError):
        pf.choose_K_kpm(mu, 0.0, 0)                # nev < 1


@pytest.mark.parametrize("D,nnz,nev,s,prec", [(924, 924 * 13, 10, 8, "f32"), (12870, 122694, 100, 32, "f64"),
                                              (184756, 2129556, 100, 32, "f32"), (853776, 11099088, 100, 64, "f32")])
def test_footprint_covers_csr_and_krylov_basis(pf, D, nnz, nev, s, prec):
    """The admission measure holds at least the CSR (int32 columns and FP64 values) and the Krylov
    basis of the expected size at eta = 1.5 (the printed fit of Sec. 5.5) for the guard count."""
    f = pf.solve_footprint(D, nnz, nev, s, prec)
    M = min(od.expected_krylov_dim(od.guard_count(nev, D), s, 1.5), D)
    assert f >= nnz * 12 + M * D * 8
    assert f >= pf.solve_footprint(D, nnz, max(1, nev // 2), s, prec)      # more pairs never need less
    assert pf.solve_footprint(D, nnz + 1000, nev, s, prec) > f


def test_footprint_errors(pf):
    with pytest.raises(pf.PolfedError):
        pf.solve_footprint(100, 500, 101, 8, "f64")    # nev > D
    with pytest.raises(pf.PolfedError):
        pf.solve_footprint(1000, 5000, 10, 12, "f64")  # block width not a power of two up to 64
    with pytest.raises(pf.PolfedError):
        pf.solve_footprint(0, 0, 1, 8, "f64")          # empty sector
