"""GPU parity of batching (a11): many problems advanced together.

Bars: the batched filter equals the one-problem filter bit for bit (same operation order
per row) and matches the oracle's Clenshaw recurrence to FP64 rounding; a batched solve
returns, for every problem, exactly what the one-problem solve returns, and both match
dense diagonalisation (eigenvalues within 1e-10 ||H||, residuals <= 1e-9 ||H||).
"""
import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh, dense, chebyshev as oc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    import paper_2605_10191_b300 as pf
    return pf


def _problems():
    # different models, sizes and degrees in one batch
    return [pi.xxz_params(10, W=1.0, seed=1101), pi.xxz_params(12, W=3.0, seed=1102),
            pi.qsun_params(N=3, L=6, seed=3101), pi.hubbard_params(5, 2, 3, U=2.0, W=2.0, seed=4101),
            pi.xxz_params(8, W=0.5, seed=1103)]


def _start(D, s, seed, dtype):
    V = pi.uniform_pm_half(seed, np.arange(D * s)).reshape(D, s)
    return torch.tensor(V, dtype=dtype, device="cuda")


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("s", [8, 32])
def test_filter_batch_bitwise_equals_single(pf, dtype, s):
    items, singles = [], []
    for j, p in enumerate(_problems()):
        H = pf.Hamiltonian.from_params(p)
        H.spectral_bounds()
        K = [40, 97, 13, 64, 1][j]
        c = pf.filter_coefficients(0.1 * j - 0.2, K)
        V = _start(H.D, s, 7 + j, dtype)
        items.append((H, V, c))
        singles.append(H.filter_apply(V, c))
    outs = pf.filter_apply_batch(items)
    torch.cuda.synchronize()
    for W, Ws in zip(outs, singles):
        assert torch.equal(W, Ws)


def test_filter_batch_matches_oracle(pf):
    items, ref = [], []
    for j, p in enumerate(_problems()[:4]):
        H = pf.Hamiltonian.from_params(p)
        H.spectral_bounds()
        Ec, dE, _, _ = H.rescaled()
        K = [30, 55, 21, 47][j]
        c = pf.filter_coefficients(0.3 - 0.2 * j, K)
        V = _start(H.D, 4, 100 + j, torch.float64)
        items.append((H, V, c))
        Ho = oh.build(p)
        Ht = oc.rescale(Ho, Ec, dE)
        ref.append(oc.clenshaw_apply(Ht, V.cpu().numpy(), c))
    outs = pf.filter_apply_batch(items)
    for (H, V, c), W, Wo in zip(items, outs, ref):
        K = len(c) - 1
        # FP64 rounding of K steps, the bar of the one-problem filter test
        assert np.abs(W.cpu().numpy() - Wo).max() <= K * 40 * 2.0 ** -53 * max(1.0, np.abs(Wo).max()) * 8


def test_filter_batch_rejects_bad_item(pf):
    p = pi.xxz_params(8, W=0.5, seed=1103)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    c = pf.filter_coefficients(0.0, 5)
    V1 = _start(H.D, 4, 1, torch.float64)
    with pytest.raises(pf.PolfedError):
        pf.filter_apply_batch([(H, V1, c), (H, _start(H.D, 4, 2, torch.float64), [])])


def _solve_problems(pf):
    specs = [(pi.xxz_params(12, W=2.0, seed=1201), 0.5, 20), (pi.xxz_params(12, W=4.0, seed=1202), 0.3, 10),
             (pi.xxz_params(10, W=1.0, seed=1203), 0.6, 8), (pi.hubbard_params(5, 2, 3, U=1.0, W=3.0, seed=4201),
                                                              0.5, 12)]
    out = []
    for p, eps, nev in specs:
        H = pf.Hamiltonian.from_params(p)
        H.spectral_bounds()
        K = H.choose_K(eps, nev)
        out.append(dict(H=H, eps=eps, nev=nev, K=K, p=p))
    return out


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_solve_batch_equals_alone_and_dense(pf, precision):
    probs = _solve_problems(pf)
    res = pf.solve_batch(probs, block=8, precision=precision, return_vectors=True)
    for pb, r in zip(probs, res):
        alone = pb["H"].solve(pb["eps"], pb["nev"], pb["K"], block=8, precision=precision)
        assert r.status == 0
        assert np.array_equal(r.evals, alone.evals)
        assert np.array_equal(r.resid, alone.resid)
        assert torch.equal(r.evecs, alone.evecs)
        assert r.report["blocks"] == alone.report["blocks"]
        assert r.report["refine_passes"] == alone.report["refine_passes"]
        Ho = oh.build(pb["p"])
        w, _ = dense.eigh_dense(Ho)
        hn = max(abs(w[0]), abs(w[-1]))
        lam = r.report["lambda_"]
        sel = dense.nearest(w, lam, pb["nev"])
        assert np.max(np.abs(r.evals - w[sel])) <= 1e-10 * hn
        assert np.max(r.resid) <= 1e-9 * hn


def test_solve_batch_mixed_precision_and_bad_item(pf):
    probs = _solve_problems(pf)[:3]
    probs[0]["precision"], probs[1]["precision"], probs[2]["precision"] = "f64", "f32", "f32"
    probs[2]["block"] = 8
    # an invalid item (nev > D) fails alone; the others finish
    probs.append(dict(H=probs[2]["H"], eps=0.5, nev=probs[2]["H"].D + 1, K=10))
    res = pf.solve_batch(probs, block=4, precision="f32")
    assert [r.status for r in res[:3]] == [0, 0, 0]
    assert res[3].status == 1   # PF_EINVAL
    for pb, r in zip(probs[:3], res[:3]):
        alone = pb["H"].solve(pb["eps"], pb["nev"], pb["K"], block=pb.get("block", 4), precision=pb["precision"],
                              return_vectors=False)
        assert np.array_equal(r.evals, alone.evals)
        assert np.array_equal(r.resid, alone.resid)


@pytest.mark.parametrize("form", ["steps", "graph", 1, 2, 4, 8, 16, "auto"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_filter_batch_forms_bitwise(pf, form, dtype):
    """Every execution form (per-step launches, CUDA graph, persistent clusters of 1-16 CTAs,
    autotuned) gives the bits of the one-problem filter."""
    items, singles = [], []
    for j, p in enumerate(_problems()):
        H = pf.Hamiltonian.from_params(p)
        H.spectral_bounds()
        K = [40, 97, 13, 64, 1][j]
        c = pf.filter_coefficients(0.1 * j - 0.2, K)
        V = _start(H.D, 8, 200 + j, dtype)
        items.append((H, V, c))
        singles.append(H.filter_apply(V, c))
    outs = pf.filter_apply_batch(items, form=form)
    torch.cuda.synchronize()
    for W, Ws in zip(outs, singles):
        assert torch.equal(W, Ws)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_filter_L18_range_form_matches_oracle_and_batch(pf, dtype):
    """At D = 48620 the FP32 step runs in the contiguous-range form; it must match the oracle
    (FP64 bar, or the FP32 error bound) and the sweep forms bit for bit."""
    p = pi.xxz_params(18, W=2.0, seed=1801)
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    Ec, dE, _, _ = H.rescaled()
    K = 40
    c = pf.filter_coefficients(0.1, K)
    V = _start(H.D, 32, 1802, dtype)
    W = H.filter_apply(V, c)
    Ht = oc.rescale(oh.build(p), Ec, dE)
    ref = oc.clenshaw_apply(Ht, V.double().cpu().numpy(), c)
    err = np.abs(W.double().cpu().numpy() - ref).max()
    if dtype == torch.float64:
        assert err <= K * 40 * 2.0 ** -53 * max(1.0, np.abs(ref).max()) * 8
    else:
        assert err < 50 * np.sqrt(K) * 2.0 ** -24 * np.abs(V.cpu().numpy()).max() * 8
    H2 = pf.Hamiltonian.from_params(pi.xxz_params(16, W=1.0, seed=1803))
    H2.spectral_bounds()
    V2 = _start(H2.D, 32, 1804, dtype)
    c2 = pf.filter_coefficients(-0.3, 25)
    W2 = H2.filter_apply(V2, c2)
    for form in ["steps", "graph"]:
        outs = pf.filter_apply_batch([(H, V, c), (H2, V2, c2)], form=form)
        assert torch.equal(outs[0], W) and torch.equal(outs[1], W2)


def test_filter_tune_reports(pf):
    small = pf.Hamiltonian.from_params(pi.xxz_params(10, W=1.0, seed=1901))
    small.spectral_bounds()
    form, us = pf.filter_tune(small, 100, s=8, precision="f32", n=1)
    assert form in (0, 1, 2, 4, 8, 16)
    assert us["raw"] > 0 and us["sweep"] > 0 and us["c1"] > 0 and us["sweep_copies"] >= 2
    # one item: the choice is the fastest measured single-item form
    cands = {0: us["raw"], **{c: us[f"c{c}"] for c in (1, 2, 4, 8, 16) if f"c{c}" in us}}
    assert cands[form] == min(cands.values())
    again, _ = pf.filter_tune(small, 100, s=8, precision="f32", n=1)
    assert again == form                                  # cached
    many, _ = pf.filter_tune(small, 100, s=8, precision="f32", n=512)
    assert many in (0, 1, 2, 4, 8, 16)
    big = pf.Hamiltonian.from_params(pi.xxz_params(20, W=1.0, seed=1902))
    big.spectral_bounds()
    f_big, us_big = pf.filter_tune(big, 100, s=32, precision="f32", n=4)
    assert f_big == 0 and "raw" not in us_big             # large shapes take the sweep, unmeasured


def test_block_autotuner(pf):
    H = pf.Hamiltonian.from_params(pi.xxz_params(14, W=2.0, seed=1951))
    H.spectral_bounds()
    s, us, cost = H.autotune_block(20, precision="f32")
    assert s in (8, 16, 32, 64) and all(v > 0 for v in us.values())
    assert cost[s] == min(cost.values())                  # the predicted cheapest width
    assert all(c <= 30 for c in cost)                     # no width above nev_g = 30
    assert H.autotune_block(20, precision="f32")[0] == s  # cached timings, same choice


def test_solve_with_autotuned_block_matches_dense(pf):
    p = pi.xxz_params(12, W=2.0, seed=1001)
    Ho = oh.build(p)
    w, _ = dense.eigh_dense(Ho)
    hn = max(abs(w[0]), abs(w[-1]))
    H = pf.Hamiltonian.from_params(p)
    H.spectral_bounds()
    s, _, _ = H.autotune_block(10, precision="f64")
    K = H.choose_K(0.5, 10)
    res = H.solve(0.5, 10, K, block=-1, precision="f64")
    assert res.status == 0 and res.report["krylov_dim"] % s == 0
    sel = dense.nearest(w, res.report["lambda_"], 10)
    assert np.max(np.abs(res.evals - w[sel])) <= 1e-10 * hn and np.max(res.resid) <= 1e-9 * hn
