"""GPU parity of the per-column-coefficient filter (pf_filter_apply_cols) and of the refinement's
residual-correction form (PF_REFINE_CORRECTION).

The correction form rests on an identity (pinned on the CPU in test_oracle_filter_lanczos.py):
P(H~) u = P(theta) u + d-recurrence on the residual r = H~ u - theta u, a Clenshaw recurrence of
degree K - 1 whose coefficients differ per column.  Here:
  * pf_filter_apply_cols against the oracle's clenshaw_apply_cols, FP64 at the FP64 filter bound
    K * 40 * u * 8 * scale, FP32 at the FP32 filter bound 50 sqrt(K) u32 8 max|V|;
  * with every column given the same coefficients it reproduces pf_filter_apply bit for bit;
  * solves with the correction form and with the direct form both return the dense oracle's
    eigenvalues nearest the target within 1e-10 ||H|| and residuals within 1e-9 ||H||, and their
    first refinement pass leaves residuals of the same size.
"""
import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh, chebyshev as oc, dense

pytestmark = pytest.mark.gpu


def _setup(p, Ec, dE):
    import paper_2605_10191_b300 as pf
    Hg = pf.Hamiltonian.from_params(p)
    Hg.set_rescale(Ec, dE)
    return Hg, oc.rescale(oh.build(p), Ec, dE)


def _coeff_table(K, s):
    return np.stack([oc.filter_coefficients(lt, K) for lt in np.linspace(-0.6, 0.7, s)], axis=1)


@pytest.mark.parametrize("K", [1, 2, 57, 300])
@pytest.mark.parametrize("s", [1, 8, 32])
def test_filter_apply_cols_f64(K, s):
    Hg, Ho = _setup(pi.xxz_params(12, W=2.0, seed=1001), -0.16, 6.72)
    V = pi.uniform_pm_half(3, np.arange(Ho.D * s)).reshape(Ho.D, s)
    C = _coeff_table(K, s)
    ref = oc.clenshaw_apply_cols(Ho, V, C)
    W = Hg.filter_apply_cols(torch.tensor(V, device="cuda"), C)
    assert np.max(np.abs(W.cpu().numpy() - ref)) <= K * 40 * 2.0 ** -53 * max(1.0, np.abs(ref).max()) * 8


@pytest.mark.parametrize("name,mk,Ec,dE", [
    ("xxz", lambda: pi.xxz_params(12, W=2.0, seed=1001), -0.16, 6.72),
    ("hubbard", lambda: pi.hubbard_params(6, 3, 3, U=1.0, W=4.0, seed=4001), 0.5, 20.0),
    ("qrem", lambda: pi.qrem_params(10, Gamma=1.0, seed=6001), 0.0, 14.0),
    ("qsun", lambda: pi.qsun_params(N=3, L=7, seed=3001), 0.0, 8.0),
])
@pytest.mark.parametrize("s", [8, 32])
def test_filter_apply_cols_f32(name, mk, Ec, dE, s):
    """FP32 through every step kernel the models use (structured XXZ and Hubbard, QREM bit flips,
    the quantum sun's CSR)."""
    Hg, Ho = _setup(mk(), Ec, dE)
    K = 300
    V = pi.uniform_pm_half(3, np.arange(Ho.D * s)).reshape(Ho.D, s)
    C = _coeff_table(K, s)
    ref = oc.clenshaw_apply_cols(Ho, V, C)
    W = Hg.filter_apply_cols(torch.tensor(V, device="cuda", dtype=torch.float32), C)
    err = np.abs(W.cpu().numpy().astype(np.float64) - ref).max()
    assert err < 50 * np.sqrt(K) * 2.0 ** -24 * np.abs(V).max() * 8, err


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("mapping", ["structured", "csr"])
def test_filter_apply_cols_uniform_equals_filter_apply(dtype, mapping):
    Hg, Ho = _setup(pi.xxz_params(12, W=2.0, seed=1001), -0.16, 6.72)
    Hg.set_mapping(mapping)
    s, K = 16, 123
    a = oc.filter_coefficients(0.05, K)
    V = torch.tensor(pi.uniform_pm_half(4, np.arange(Ho.D * s)).reshape(Ho.D, s), device="cuda", dtype=dtype)
    W1 = Hg.filter_apply(V, a)
    W2 = Hg.filter_apply_cols(V, np.repeat(a[:, None], s, axis=1))
    assert torch.equal(W1, W2)


@pytest.mark.parametrize("name,mk,nev,s,eps", [
    ("xxz12", lambda: pi.xxz_params(12, W=2.0, seed=1001), 20, 8, 0.5),
    ("xxz14", lambda: pi.xxz_params(14, W=3.0, seed=1401), 40, 16, 0.4),
    ("hubbard7", lambda: pi.hubbard_params(7, 3, 3, U=1.0, W=4.0, seed=4002), 16, 8, 0.5),
    ("qsun8", lambda: pi.qsun_params(N=3, L=8, seed=3002), 16, 8, 0.55),
])
def test_solve_correction_and_direct_forms_match_dense(name, mk, nev, s, eps):
    import paper_2605_10191_b300 as pf
    p = mk()
    w, _ = dense.eigh_dense(oh.build(p))
    hn = max(abs(w[0]), abs(w[-1]))
    lam = w[0] + eps * (w[-1] - w[0])
    sel = dense.nearest(w, lam, nev)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    K = H.choose_K(eps, nev)
    out = {}
    for form in ("correction", "direct"):
        r = H.solve(eps, nev, K, block=s, precision="f32", target_abs=lam, refine_form=form)
        assert r.status == 0, form
        assert np.max(np.abs(r.evals - w[sel])) <= 1e-10 * hn, form
        assert np.max(r.resid) <= 1e-9 * hn, form
        out[form] = r.report
    rc, rd = out["correction"], out["direct"]
    if rc["refine_passes"] and rd["refine_passes"]:
        a, b = rc["refine_residual"][0], rd["refine_residual"][0]
        assert 0.5 * b <= a <= 2.0 * b, (a, b)


def test_correction_form_is_the_default_with_fp64_refinement():
    """The default refinement (refine_precision FP64, refine_form 0) takes the correction form: its
    FP64 work is one step per refined block and pass; the direct form runs K FP64 steps."""
    import paper_2605_10191_b300 as pf
    H = pf.Hamiltonian.from_params(pi.xxz_params(14, W=3.0, seed=1401))
    H.spectral_bounds()
    K = H.choose_K(0.5, 40)
    r0 = H.solve(0.5, 40, K, block=16, precision="f32", return_vectors=False)
    rd = H.solve(0.5, 40, K, block=16, precision="f32", return_vectors=False, refine_form="direct")
    if rd.report["refine_passes"] == 0:
        pytest.skip("no refinement pass needed")
    blocks = sum(rd.report["refine_active"][:rd.report["refine_passes"]])
    assert rd.report["filter_steps_f64"] >= blocks * 2
    passes_blocks = sum(r0.report["refine_active"][:r0.report["refine_passes"]])
    assert r0.report["filter_steps_f64"] == passes_blocks
