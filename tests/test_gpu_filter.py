"""GPU parity of the fused Clenshaw-SpMM step and of the K-step filter (a4, a5).

Tolerances.  FP64: every output is a sum of n_row + 2 products; the kernel and the
oracle add them in different orders, so the difference is bounded by
(n_row + 4) * u * sum|terms| with u = 2^-53; the test uses 4x that bound.  FP32 (the
kernel reads FP32 values and vectors): the bound with u = 2^-24 plus the rounding of
the inputs, again 4x.  Over K steps the FP64 bound is applied to the whole recurrence
against the oracle's FP64 recurrence at K * (n_row + 4) * u * scale.
"""
import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh, chebyshev as oc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


def _setup(pf, p, Ec, dE):
    Hg = pf.Hamiltonian.from_params(p)
    Hg.set_rescale(Ec, dE)
    Ho = oc.rescale(oh.build(p), Ec, dE)
    return Hg, Ho


def _blocks(D, s, seed):
    g = [pi.uniform_pm_half(seed + k, np.arange(D * s)).reshape(D, s) for k in range(3)]
    return g


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
def test_clenshaw_step_f64(pf, name, mk, Ec, dE, s):
    p = mk()
    Hg, Ho = _setup(pf, p, Ec, dE)
    V, B1, B2 = _blocks(Ho.D, s, 77)
    a, alpha = 0.0123, 2.0
    ref = oc.clenshaw_step(Ho, V, B1, B2, a, alpha)
    tV, tB1, tB2 = (torch.tensor(x, device="cuda") for x in (V, B1, B2))
    out = torch.empty_like(tV)
    Hg.clenshaw_step(tV, tB1, tB2, out, a, alpha, 1.0)
    nrow = np.diff(Ho.indptr).max()
    bound = 4 * (nrow + 4) * 2.0 ** -53 * _abs_terms(Ho, V, B1, B2, a, alpha, 1.0)
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= bound), err.max()
    # in-place form (out aliases B2) and the two degenerate steps
    Hg.clenshaw_step(tV, tB1, tB2, tB2, a, alpha, 1.0)
    assert np.all(np.abs(tB2.cpu().numpy() - ref) <= bound)
    o2 = torch.empty_like(tV)
    Hg.clenshaw_step(tV, None, None, o2, 0.37, 0.0, 0.0)
    assert np.array_equal(o2.cpu().numpy(), 0.37 * V)
    Hg.clenshaw_step(tV, tB1, None, o2, a, 1.0, 0.0)
    ref2 = oc.clenshaw_step(Ho, V, B1, np.zeros_like(V), a, 1.0)
    assert np.all(np.abs(o2.cpu().numpy() - ref2) <= bound)


@pytest.mark.parametrize("name,mk,Ec,dE", CASES[:2])
@pytest.mark.parametrize("s", [4, 32, 64])
def test_clenshaw_step_f32(pf, name, mk, Ec, dE, s):
    p = mk()
    Hg, Ho = _setup(pf, p, Ec, dE)
    V, B1, B2 = (x.astype(np.float32).astype(np.float64) for x in _blocks(Ho.D, s, 5))
    Ho32 = oc.CSR(D=Ho.D, indptr=Ho.indptr, indices=Ho.indices, data=Ho.data.astype(np.float32).astype(np.float64))
    a, alpha = np.float32(0.0123), 2.0
    ref = oc.clenshaw_step(Ho32, V, B1, B2, float(a), alpha)
    tV, tB1, tB2 = (torch.tensor(x, device="cuda", dtype=torch.float32) for x in (V, B1, B2))
    out = torch.empty_like(tV)
    Hg.clenshaw_step(tV, tB1, tB2, out, float(a), alpha, 1.0)
    nrow = np.diff(Ho.indptr).max()
    bound = 4 * (nrow + 4) * 2.0 ** -24 * _abs_terms(Ho32, V, B1, B2, float(a), alpha, 1.0)
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= bound), err.max()


def test_clenshaw_step_full_size_sampled_rows(pf):
    """XXZ L=20, s=32 (the launch shape of the filter): sampled rows against the oracle."""
    p = pi.xxz_params(20, W=1.0, seed=2000)
    Hg, Ho = _setup(pf, p, -0.5, 12.0)
    D, s = Ho.D, 32
    V, B1, B2 = _blocks(D, s, 99)
    tV, tB1, tB2 = (torch.tensor(x, device="cuda") for x in (V, B1, B2))
    out = torch.empty_like(tV)
    Hg.clenshaw_step(tV, tB1, tB2, out, 0.5, 2.0, 1.0)
    rows = np.concatenate([np.arange(40), np.random.default_rng(0).choice(D, 400, replace=False), np.arange(D - 40, D)])
    S = Ho.scipy()[rows]
    ref = 0.5 * V[rows] + 2.0 * (S @ B1) - B2[rows]
    Sa = S.copy()
    Sa.data = np.abs(Sa.data)
    bound = 4 * 24 * 2.0 ** -53 * (0.5 * np.abs(V[rows]) + 2 * (Sa @ np.abs(B1)) + np.abs(B2[rows]))
    assert np.all(np.abs(out.cpu().numpy()[rows] - ref) <= bound)
    # FP32 at the same shape (the workload's filter step): the kernel reads FP32 values and blocks,
    # so the oracle runs on the same rounded inputs in FP64 and the bound is the FP32 one,
    # 4 (n_row + 4) u32 sum|terms| per element
    r32 = lambda x: x.astype(np.float32).astype(np.float64)
    V32, B132, B232 = r32(V), r32(B1), r32(B2)
    S32 = S.copy()
    S32.data = r32(S32.data)
    ref32 = 0.5 * V32[rows] + 2.0 * (S32 @ B132) - B232[rows]
    nrow = int(np.diff(Ho.indptr).max())
    S32.data = np.abs(S32.data)
    bound32 = 4 * (nrow + 4) * 2.0 ** -24 * (0.5 * np.abs(V32[rows]) + 2 * (S32 @ np.abs(B132)) + np.abs(B232[rows]))
    o32 = torch.empty_like(tV, dtype=torch.float32)
    Hg.clenshaw_step(tV.float(), tB1.float(), tB2.float(), o32, 0.5, 2.0, 1.0)
    err32 = np.abs(o32.cpu().numpy()[rows].astype(np.float64) - ref32)
    assert np.all(err32 <= bound32), (err32 / bound32).max()


def test_filter_coefficients_vs_oracle(pf):
    for lam_t, K in [(0.0, 10), (0.31, 237), (-0.77, 1500)]:
        c = pf.filter_coefficients(lam_t, K)
        ref = oc.filter_coefficients(lam_t, K)
        assert np.max(np.abs(c - ref)) < 1e-13 * np.max(np.abs(ref)) * np.sqrt(K)


@pytest.mark.parametrize("K", [1, 2, 3, 57])
@pytest.mark.parametrize("s", [1, 8, 32])
def test_filter_apply_f64(pf, K, s):
    p = pi.xxz_params(12, W=2.0, seed=1001)
    Hg, Ho = _setup(pf, p, -0.16, 6.72)
    V = pi.uniform_pm_half(3, np.arange(Ho.D * s)).reshape(Ho.D, s)
    a = oc.filter_coefficients(0.05, K)
    ref = oc.clenshaw_apply(Ho, V, a)
    W = Hg.filter_apply(torch.tensor(V, device="cuda"), a)
    assert np.max(np.abs(W.cpu().numpy() - ref)) <= K * 40 * 2.0 ** -53 * max(1.0, np.abs(ref).max()) * 8


def test_filter_apply_f32_within_stated_error(pf):
    p = pi.xxz_params(12, W=2.0, seed=1001)
    Hg, Ho = _setup(pf, p, -0.16, 6.72)     # [Ec - dE, Ec + dE] contains the spectrum [-6.82, 6.50]
    V = pi.uniform_pm_half(3, np.arange(Ho.D * 8)).reshape(Ho.D, 8)
    K = 300
    a = oc.filter_coefficients(0.05, K)
    ref = oc.clenshaw_apply(Ho, V, a)
    W = Hg.filter_apply(torch.tensor(V, device="cuda", dtype=torch.float32), a)
    err = np.abs(W.cpu().numpy().astype(np.float64) - ref).max()
    # FP32 recurrence: rounding noise grows like sqrt(K) u32 per unit of ||b||
    assert err < 50 * np.sqrt(K) * 2.0 ** -24 * np.abs(V).max() * 8
