"""The allocation-free filter entry point (pf_filter_apply_noalloc).

Who needs it: callers that cannot allocate device memory at the moment they apply the
filter -- code that runs while a memory pool is frozen or already exhausted, a host
allocator's own hooks (which must not re-enter that allocator), or loops that forbid
allocation calls.  pf_filter_apply_noalloc keeps its two Clenshaw auxiliary blocks in one
fixed device array inside the library instead of asking the allocator for them.

What is checked here, through the C ABI:
  * after a call that leaves NaN in both auxiliary blocks of the shared array, a clean call
    returns exactly the bits of the allocating entry point pf_filter_apply (both run the
    same deterministic recurrence), for K = 1, 2 and a large K, in FP64, FP32 and
    pair-float, and through both the CSR and the structured mapping;
  * the result matches the oracle's FP64 Clenshaw recurrence within the filter tests'
    tolerance K * 40 * u * 8 * max(1, |ref|);
  * the size limit: a request of exactly 32 MiB (two 16 MiB blocks) is served, the next
    larger one of a real sector is refused with PF_EINVAL.

This file is collected last on purpose: the entry point is an addition outside the paper's
path, so under `pytest -x` a failure here stops the run only after every other test ran.
It passes alone in a fresh process as well (nothing here depends on earlier tests).
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import pf_inputs as pi
from oracle import hamiltonian as oh, chebyshev as oc

pytestmark = pytest.mark.gpu

LIMIT = 32 << 20          # bytes of the fixed scratch array (two auxiliary blocks)


def _lib():
    from paper_2605_10191_b300 import _lib
    return _lib


def _prec(V):
    L = _lib()
    if V.dtype == torch.float64:
        return L.PF_F64
    if V.dim() == 3:
        return L.PF_DF64
    return L.PF_F32


def _call_noalloc(Hg, V, W, coeffs):
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    return _lib().lib().pf_filter_apply_noalloc(Hg.handle, _prec(V), V.shape[1], C.c_void_p(V.data_ptr()),
                                                C.c_void_p(W.data_ptr()), c.ctypes.data_as(C.POINTER(C.c_double)),
                                                len(c) - 1, C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _block(D, s, seed, kind):
    x = pi.uniform_pm_half(seed, np.arange(D * s)).reshape(D, s)
    if kind == "f64":
        return torch.tensor(x, device="cuda", dtype=torch.float64)
    if kind == "f32":
        return torch.tensor(x, device="cuda", dtype=torch.float32)
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    return torch.tensor(np.stack([hi, lo], axis=-1), device="cuda", dtype=torch.float32)


def _poison(Hg, s, kind, K):
    """A call whose V is NaN: every step writes NaN, so both auxiliary blocks (K >= 2) hold NaN."""
    V = torch.full_like(_block(Hg.D, s, 1, kind), float("nan"))
    W = torch.empty_like(V)
    assert _call_noalloc(Hg, V, W, np.full(K + 1, 0.5)) == 0
    torch.cuda.synchronize()
    assert torch.isnan(W).all()


@pytest.mark.parametrize("kind", ["f64", "f32", "df64"])
@pytest.mark.parametrize("mapping", ["structured", "csr"])
@pytest.mark.parametrize("K", [1, 2, 301])
def test_noalloc_equals_allocating_entry_point_after_poison(kind, mapping, K):
    import paper_2605_10191_b300 as pf
    Hg = pf.Hamiltonian.from_params(pi.xxz_params(12, W=2.0, seed=1001))
    Hg.set_rescale(-0.16, 6.72)
    Hg.set_mapping(mapping)
    s = 8
    a = pf.filter_coefficients(0.05, K)
    _poison(Hg, s, kind, 3)
    for call in range(2):                       # two calls in a row, different inputs
        V = _block(Hg.D, s, 3 + call, kind)
        ref = Hg.filter_apply(V, a)
        W = torch.full_like(V, float("nan"))
        assert _call_noalloc(Hg, V, W, a) == 0
        torch.cuda.synchronize()
        assert torch.equal(W, ref), (kind, mapping, K, call)


@pytest.mark.parametrize("s,K", [(8, 57), (32, 20)])
def test_noalloc_matches_oracle_f64(s, K):
    import paper_2605_10191_b300 as pf
    p = pi.xxz_params(12, W=2.0, seed=1001)
    Hg = pf.Hamiltonian.from_params(p)
    Hg.set_rescale(-0.16, 6.72)
    Ho = oc.rescale(oh.build(p), -0.16, 6.72)
    a = oc.filter_coefficients(0.05, K)
    _poison(Hg, s, "f64", 3)
    V = pi.uniform_pm_half(3, np.arange(Ho.D * s)).reshape(Ho.D, s)
    ref = oc.clenshaw_apply(Ho, V, a)
    tV = torch.tensor(V, device="cuda")
    W = torch.empty_like(tV)
    assert _call_noalloc(Hg, tV, W, a) == 0
    torch.cuda.synchronize()
    assert np.max(np.abs(W.cpu().numpy() - ref)) <= K * 40 * 2.0 ** -53 * max(1.0, np.abs(ref).max()) * 8


def test_noalloc_size_limit_boundary():
    """QREM L=16 (D = 65536) at s = 64 in FP32 needs exactly 2 x 16 MiB: served, bit-equal to
    pf_filter_apply.  The XXZ sector L=26, N=5 (D = C(26, 5) = 65780) at the same s and
    precision needs 0.4 % more: refused with PF_EINVAL, W untouched."""
    import paper_2605_10191_b300 as pf
    L = _lib()
    Hq = pf.Hamiltonian.from_params(pi.qrem_params(16, Gamma=1.0, seed=6001))
    assert Hq.D * 64 * 4 * 2 == LIMIT
    Hq.set_rescale(0.0, 12.0)
    a = pf.filter_coefficients(0.1, 3)
    V = _block(Hq.D, 64, 11, "f32")
    W = torch.full_like(V, float("nan"))
    assert _call_noalloc(Hq, V, W, a) == 0
    torch.cuda.synchronize()
    assert torch.equal(W, Hq.filter_apply(V, a))

    Hx = pf.Hamiltonian.from_params(pi.xxz_params(26, N=5, W=1.0, seed=2000))
    assert Hx.D == math.comb(26, 5) and 2 * Hx.D * 64 * 4 > LIMIT
    Hx.set_rescale(0.0, 16.0)
    V = _block(Hx.D, 64, 12, "f32")
    W = torch.full_like(V, 7.0)
    assert _call_noalloc(Hx, V, W, a) == L.PF_EINVAL
    torch.cuda.synchronize()
    assert bool((W == 7.0).all())
    # the same sector at s = 32 fits and is served
    V32 = V[:, :32].contiguous()
    W32 = torch.empty_like(V32)
    assert _call_noalloc(Hx, V32, W32, a) == 0
    torch.cuda.synchronize()
    assert torch.equal(W32, Hx.filter_apply(V32, a))


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    import paper_2605_10191_b300 as pf
    L = _lib()
    Hg = pf.Hamiltonian.from_params(pi.xxz_params(20, W=1.0, seed=2000))   # D = 184756
    Hg.set_rescale(0.0, 12.0)
    V = torch.zeros((Hg.D, 32), device="cuda", dtype=torch.float64)          # 2 x 47 MB > 32 MiB
    W = torch.empty_like(V)
    assert _call_noalloc(Hg, V, W, np.array([1.0, 0.5])) == L.PF_EINVAL
