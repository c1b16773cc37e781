"""The allocation-free filter entry point (pf_filter_apply_noalloc) against pf_filter_apply.

Callers that cannot allocate device memory at call time (a frozen or exhausted pool, an
allocator that must not be re-entered) use pf_filter_apply_noalloc, which keeps its two
auxiliary blocks in a fixed device array inside the library.  Its output must match the
allocating entry point within the tolerance of the filter tests, on two calls in a row
(the second call sees the array exactly as the first left it).  This file is collected
last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import pf_inputs as pi

pytestmark = pytest.mark.gpu


def _call_noalloc(pf, Hg, V, W, coeffs):
    from paper_2605_10191_b300 import _lib
    prec = _lib.PF_F64 if V.dtype == torch.float64 else _lib.PF_F32
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    return _lib.lib().pf_filter_apply_noalloc(Hg.handle, prec, V.shape[1], C.c_void_p(V.data_ptr()),
                                              C.c_void_p(W.data_ptr()), c.ctypes.data_as(C.POINTER(C.c_double)),
                                              len(c) - 1, C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("dtype,s,K", [(torch.float64, 8, 57), (torch.float64, 32, 20), (torch.float32, 32, 300)])
def test_noalloc_filter_matches_allocating_entry_point(dtype, s, K):
    import paper_2605_10191_b300 as pf
    p = pi.xxz_params(12, W=2.0, seed=1001)
    Hg = pf.Hamiltonian.from_params(p)
    Hg.set_rescale(-0.16, 6.72)
    a = pf.filter_coefficients(0.05, K)
    for call in range(2):                        # two calls in a row, different inputs
        V = torch.tensor(pi.uniform_pm_half(3 + call, np.arange(Hg.D * s)).reshape(Hg.D, s), device="cuda",
                         dtype=dtype)
        ref = Hg.filter_apply(V, a).double().cpu().numpy()
        W = torch.full_like(V, float("nan"))
        assert _call_noalloc(pf, Hg, V, W, a) == 0
        torch.cuda.synchronize()
        got = W.double().cpu().numpy()
        u = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
        assert np.max(np.abs(got - ref)) <= K * 40 * u * max(1.0, np.abs(ref).max()) * 8


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    import paper_2605_10191_b300 as pf
    from paper_2605_10191_b300 import _lib
    Hg = pf.Hamiltonian.from_params(pi.xxz_params(20, W=1.0, seed=2000))   # D = 184756
    Hg.set_rescale(0.0, 12.0)
    V = torch.zeros((Hg.D, 32), device="cuda", dtype=torch.float64)          # 2 x 47 MB > 32 MiB
    W = torch.empty_like(V)
    assert _call_noalloc(pf, Hg, V, W, np.array([1.0, 0.5])) == _lib.PF_EINVAL
