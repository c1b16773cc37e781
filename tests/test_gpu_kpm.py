"""GPU parity of the kernel-polynomial density of states (Sec. 3.3, App. B).

Bars: the device moments equal the oracle's (same random block) to FP64 rounding; the density,
the :maxdos / offset targets and K from Eq. condition_for_K equal the oracle's on the same
moments; a solve at the :maxdos target returns the dense oracle's nearest eigenvalues.
"""
import numpy as np
import pytest

import pf_inputs as pi
from oracle import hamiltonian as oh, chebyshev as oc, dense, kpm, dos as od

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


@pytest.fixture(scope="module")
def setup(pf):
    p = pi.xxz_params(12, W=2.0, seed=1001)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    Ec, dE, _, _ = H.rescaled()
    Ht = oc.rescale(oh.build(p), Ec, dE)
    return p, H, Ht, Ec, dE


@pytest.mark.parametrize("N,R", [(64, 8), (33, 1), (128, 32)])
def test_kpm_moments_match_oracle(pf, setup, N, R):
    p, H, Ht, Ec, dE = setup
    mu = H.kpm_moments(N=N, R=R, seed=4242)
    ref = kpm.moments(Ht, kpm.random_block(H.D, R, 4242), N)
    assert np.max(np.abs(mu - ref)) <= 1e-9 * H.D


def test_kpm_dos_target_and_K_match_oracle(pf, setup):
    p, H, Ht, Ec, dE = setup
    mu = H.kpm_moments(N=96, R=16, seed=9)
    x = np.linspace(-0.95, 0.95, 77)
    assert np.max(np.abs(pf.kpm_dos(mu, x) - kpm.dos_kpm(x, mu))) <= 1e-10 * H.D
    em = kpm.maxdos(mu)
    assert abs(pf.kpm_target(mu, 0.0) - em) < 1e-12
    for eta in (-0.6, 0.3, 1.0):
        assert abs(pf.kpm_target(mu, eta) - kpm.offset_target(em, eta)) < 1e-12
    for lam_t, nev in ((em, 20), (0.2, 10), (-0.4, 30)):
        assert pf.choose_K_kpm(mu, lam_t, nev) == kpm.choose_K(lam_t, od.guard_count(nev, mu[0]), mu)


def test_solve_at_maxdos_target(pf, setup):
    p, H, Ht, Ec, dE = setup
    mu = H.kpm_moments(N=96, R=16, seed=11)
    lam_t = pf.kpm_target(mu, 0.0)
    K = pf.choose_K_kpm(mu, lam_t, 16)
    lam = H.target_abs(lam_t)
    res = H.solve(0.5, 16, K, block=8, precision="f64", target_abs=lam)
    w, _ = dense.eigh_dense(oh.build(p))
    hn = max(abs(w[0]), abs(w[-1]))
    sel = dense.nearest(w, lam, 16)
    assert res.status == 0
    assert np.max(np.abs(res.evals - w[sel])) <= 1e-10 * hn
    assert np.max(res.resid) <= 1e-9 * hn


def test_kpm_errors(pf, setup):
    p, H, Ht, Ec, dE = setup
    with pytest.raises(pf.PolfedError):
        H.kpm_moments(N=16, R=3)                        # R not a power of two
    with pytest.raises(pf.PolfedError):
        pf.kpm_target(np.ones(8), 1.5)                  # eta outside [-1, 1]
    with pytest.raises(pf.PolfedError):
        pf.kpm_dos(np.ones(8), [1.0])                   # x on the edge
