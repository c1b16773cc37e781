"""GPU parity of the pair-float (PF_DF64) Clenshaw step, filter and refinement.

A pair-float entry is (hi, lo), value hi + lo, two floats.  The kernel reads H~ and the
blocks as pairs, so the oracle is run on exactly the values the pairs hold (the FP64
inputs rounded to pairs here, on the host).

Tolerance, from the arithmetic: a product x y loses at most x.lo y.lo plus the roundings of
three FMAs on terms of size <= 2^-23 |x y|, under 6 * 2^-48 |x y|; each of the n additions
of a row adds one rounding of the low word, whose size stays below n * 2^-24 sum|terms|,
so a row is within (n + 6) * 2^-47 sum|terms|.  The tests use 4 x (n_row + 8) * 2^-46
sum|terms| per step (about 1e-12 relative: far below FP32's 2^-24, which a dropped low
word would show) and K times that over a K-step recurrence, as the FP64 tests do.
"""
import dataclasses

import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh, chebyshev as oc, dense

pytestmark = pytest.mark.gpu

U_DF = 2.0 ** -46


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


def to_pair(x):
    """FP64 array -> float32 array with a trailing (hi, lo) axis."""
    x = np.asarray(x, dtype=np.float64)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return np.stack([hi, lo], axis=-1)


def from_pair(p):
    p = np.asarray(p)
    return p[..., 0].astype(np.float64) + p[..., 1].astype(np.float64)


def _dev(p):
    return torch.tensor(p, dtype=torch.float32, device="cuda")


def _setup(pf, p, Ec, dE):
    Hg = pf.Hamiltonian.from_params(p)
    Hg.set_rescale(Ec, dE)
    Ho = oc.rescale(oh.build(p), Ec, dE)
    Hp = dataclasses.replace(Ho, data=from_pair(to_pair(Ho.data)))   # the values the kernel reads
    return Hg, Ho, Hp


def _abs_terms(Ho, V, B1, B2, a, alpha, beta):
    S = Ho.scipy().copy()
    S.data = np.abs(S.data)
    return np.abs(a * V) + abs(alpha) * (S @ np.abs(B1)) + abs(beta) * np.abs(B2)


CASES = [
    ("xxz12", lambda: pi.xxz_params(12, W=2.0, seed=1001), 0.1, 7.0),
    ("xxz16", lambda: pi.xxz_params(16, W=3.0, seed=7), -0.2, 9.0),
    ("qsun", lambda: pi.qsun_params(N=3, L=9, seed=3), 0.0, 6.0),
    ("hubbard", lambda: pi.hubbard_params(6, 3, 3, U=1.0, W=4.0, seed=4001), 0.5, 20.0),
]


@pytest.mark.parametrize("name,mk,Ec,dE", CASES)
@pytest.mark.parametrize("s", [1, 2, 4, 8, 16, 32, 64])
def test_clenshaw_step_df64(pf, name, mk, Ec, dE, s):
    Hg, Ho, Hp = _setup(pf, mk(), Ec, dE)
    D = Ho.D
    blocks = [to_pair(pi.uniform_pm_half(77 + k, np.arange(D * s)).reshape(D, s)) for k in range(3)]
    V, B1, B2 = (from_pair(b) for b in blocks)
    a, alpha = 0.0123, 2.0
    ap = from_pair(to_pair(a))
    ref = oc.clenshaw_step(Hp, V, B1, B2, ap, alpha)
    tV, tB1, tB2 = (_dev(b) for b in blocks)
    out = torch.empty_like(tV)
    Hg.clenshaw_step(tV, tB1, tB2, out, a, alpha, 1.0)
    nrow = np.diff(Ho.indptr).max()
    bound = 4 * (nrow + 8) * U_DF * _abs_terms(Hp, V, B1, B2, ap, alpha, 1.0)
    got = out.cpu().numpy()
    assert np.all(np.abs(from_pair(got) - ref) <= bound), np.abs(from_pair(got) - ref).max()
    # stored pairs are normalised: |lo| <= half an ulp of hi
    hi, lo = got[..., 0], got[..., 1]
    assert np.all(np.abs(lo) <= np.spacing(np.abs(hi)) / 2)
    # in place (out aliases B2) gives the same bits; the degenerate steps
    Hg.clenshaw_step(tV, tB1, tB2, tB2, a, alpha, 1.0)
    assert torch.equal(tB2, out)
    o2 = torch.empty_like(tV)
    Hg.clenshaw_step(tV, None, None, o2, 0.37, 0.0, 0.0)
    a37 = from_pair(to_pair(0.37))
    assert np.all(np.abs(from_pair(o2.cpu().numpy()) - a37 * V) <= 4 * U_DF * np.abs(a37 * V))
    Hg.clenshaw_step(tV, tB1, None, o2, a, 1.0, 0.0)
    ref2 = oc.clenshaw_step(Hp, V, B1, np.zeros_like(V), ap, 1.0)
    assert np.all(np.abs(from_pair(o2.cpu().numpy()) - ref2) <= bound)


@pytest.mark.parametrize("name,mk,Ec,dE", CASES)
@pytest.mark.parametrize("s,K", [(8, 40), (32, 97), (4, 1), (16, 2)])
def test_filter_df64_matches_oracle(pf, name, mk, Ec, dE, s, K):
    # The recurrence is run as the solve runs it, with the spectrum of H~ inside [-1, 1]
    # (bounds from pf_spectral_bounds), so |b_i| <= (K + 1) max|a| ||V||.  A pair has FP32's
    # exponent range: a recurrence grown past 3.4e38 (a spectrum outside [-1, 1] and large K)
    # overflows, where FP64 would not.
    p = mk()
    Hg = pf.Hamiltonian.from_params(p)
    Hg.spectral_bounds()
    Ec, dE, _, _ = Hg.rescaled()
    Ho = oc.rescale(oh.build(p), Ec, dE)
    Hp = dataclasses.replace(Ho, data=from_pair(to_pair(Ho.data)))
    D = Ho.D
    Vp = to_pair(pi.uniform_pm_half(91, np.arange(D * s)).reshape(D, s))
    c = pf.filter_coefficients(0.13, K)
    cp = from_pair(to_pair(c))
    ref = oc.clenshaw_apply(Hp, from_pair(Vp), cp)
    W = Hg.filter_apply(_dev(Vp), c)
    nrow = np.diff(Ho.indptr).max()
    scale = max(1.0, np.abs(ref).max(), np.abs(from_pair(Vp)).max())
    err = np.abs(from_pair(W.cpu().numpy()) - ref).max()
    assert err <= 8 * (K + 1) * (nrow + 8) * U_DF * scale, err
    # and it is FP64-class: within the FP64 filter's own distance of the FP64 oracle, x 64
    W64 = Hg.filter_apply(torch.tensor(from_pair(Vp), device="cuda"), c)
    ref64 = oc.clenshaw_apply(Ho, from_pair(Vp), c)
    d64 = np.abs(W64.cpu().numpy() - ref64).max()
    assert np.abs(from_pair(W.cpu().numpy()) - ref64).max() <= max(64 * d64, 8 * (K + 1) * (nrow + 8) * U_DF * scale)


def _problems():
    return [pi.xxz_params(10, W=1.0, seed=1101), pi.xxz_params(12, W=3.0, seed=1102),
            pi.qsun_params(N=3, L=6, seed=3101), pi.hubbard_params(5, 2, 3, U=2.0, W=2.0, seed=4101),
            pi.xxz_params(8, W=0.5, seed=1103)]


@pytest.mark.parametrize("form", ["steps", "graph", 1, 2, 4, 8, 16, "auto"])
@pytest.mark.parametrize("s", [8, 32])
def test_filter_df64_forms_bitwise(pf, form, s):
    """Every execution form gives the bits of the one-problem pair-float filter."""
    items, singles = [], []
    for j, p in enumerate(_problems()):
        H = pf.Hamiltonian.from_params(p)
        H.spectral_bounds()
        K = [40, 97, 13, 64, 1][j]
        c = pf.filter_coefficients(0.1 * j - 0.2, K)
        V = _dev(to_pair(pi.uniform_pm_half(300 + j, np.arange(H.D * s)).reshape(H.D, s)))
        items.append((H, V, c))
        singles.append(H.filter_apply(V, c))
    outs = pf.filter_apply_batch(items, form=form)
    torch.cuda.synchronize()
    for W, Ws in zip(outs, singles):
        assert torch.equal(W, Ws)


def test_filter_df64_L18_range_form(pf):
    """D = 48620: the pair-float step runs in the contiguous-range form; it matches the oracle
    and the sweep forms bit for bit."""
    p = pi.xxz_params(18, W=2.0, seed=1801)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    Ec, dE, _, _ = H.rescaled()
    K = 40
    c = pf.filter_coefficients(0.1, K)
    Vp = to_pair(pi.uniform_pm_half(1802, np.arange(H.D * 32)).reshape(H.D, 32))
    W = H.filter_apply(_dev(Vp), c)
    Ht = oc.rescale(oh.build(p), Ec, dE)
    Ht.data = from_pair(to_pair(Ht.data))
    ref = oc.clenshaw_apply(Ht, from_pair(Vp), from_pair(to_pair(c)))
    err = np.abs(from_pair(W.cpu().numpy()) - ref).max()
    assert err <= 8 * (K + 1) * 40 * U_DF * max(1.0, np.abs(ref).max()), err
    H2 = pf.Hamiltonian.from_params(pi.xxz_params(16, W=1.0, seed=1803))
    H2.spectral_bounds()
    V2 = _dev(to_pair(pi.uniform_pm_half(1804, np.arange(H2.D * 32)).reshape(H2.D, 32)))
    c2 = pf.filter_coefficients(-0.3, 25)
    W2 = H2.filter_apply(V2, c2)
    for form in ["steps", "graph"]:
        outs = pf.filter_apply_batch([(H, _dev(Vp), c), (H2, V2, c2)], form=form)
        assert torch.equal(outs[0], W) and torch.equal(outs[1], W2)


@pytest.mark.parametrize("L,nev,s", [(12, 20, 8), (14, 40, 16)])
def test_solve_refine_pairfloat_vs_fp64(pf, L, nev, s):
    """FP32 filter with the refinement in pair-float or in FP64: both reach the residual bar
    and the dense eigenvalues; FP64 is the default."""
    p = pi.xxz_params(L, W=2.5, seed=2200 + L)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    K = H.choose_K(0.5, nev)
    w, _ = dense.eigh_dense(oh.build(p))
    hn = max(abs(w[0]), abs(w[-1]))
    lam = w[0] + 0.5 * (w[-1] - w[0])
    sel = dense.nearest(w, lam, nev)
    out = {}
    for rp in ("df64", "f64"):
        r = H.solve(0.5, nev, K, block=s, precision="f32", target_abs=lam, refine_precision=rp)
        assert r.status == 0, rp
        assert r.report["refine_passes"] >= 1
        assert np.max(np.abs(r.evals - w[sel])) <= 1e-10 * hn, rp
        assert np.max(r.resid) <= 1e-9 * hn, rp
        out[rp] = r
    d = H.solve(0.5, nev, K, block=s, precision="f32", target_abs=lam)
    assert np.array_equal(d.evals, out["f64"].evals)


def test_pairfloat_rejects(pf):
    H = pf.Hamiltonian.from_params(pi.xxz_params(8, W=1.0, seed=5))
    H.spectral_bounds()
    with pytest.raises(pf.PolfedError):
        H.solve(0.5, 4, 20, block=4, precision="f32", refine_precision=1)   # PF_F32 is not a refinement arithmetic
    V = torch.zeros(H.D, 4, 2, device="cuda")
    with pytest.raises(pf.PolfedError):   # the unscaled H is FP64 only
        H.clenshaw_step(V, V, None, torch.empty_like(V), 0.0, 1.0, 0.0, use_H=True)
