"""Python binding of libpolfed (argument marshalling only; every step runs in the CUDA library).

PyTorch supplies device memory (through the allocator hook) and streams.  Vector
blocks are torch tensors of shape (D, s), row-major, float64 or float32, on the
current CUDA device; a pair-float block (PF_DF64) is a float32 tensor of shape
(D, s, 2) holding (hi, lo) per entry.
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from ._lib import check, lib

_ALLOC_REFS = []


def _install_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    if _ALLOC_REFS:
        return

    def _alloc(ctx, nbytes, stream):
        try:
            dev = torch.cuda.current_device()
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream or None))
        except Exception:
            return None

    def _free(ctx, ptr, stream):
        if ptr:
            torch.cuda.caching_allocator_delete(ptr)

    a, f = L.ALLOC_FN(_alloc), L.FREE_FN(_free)
    _ALLOC_REFS.extend([a, f])
    check(lib().pf_set_allocator(a, f, None), "pf_set_allocator")


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _block_prec(V):
    """Filter precision of a vector block: float64 (D, s), float32 (D, s) or pairs (D, s, 2)."""
    if V.dtype == torch.float64:
        return L.PF_F64
    if V.dtype == torch.float32 and V.dim() == 3 and V.shape[2] == 2:
        return L.PF_DF64
    return L.PF_F32


_PREC_NAMES = {"f64": L.PF_F64, "f32": L.PF_F32, "df64": L.PF_DF64}


_REFINE_FORMS = {"default": 0, "direct": L.PF_REFINE_DIRECT, "correction": L.PF_REFINE_CORRECTION}


def _refine_form_code(name):
    if name not in _REFINE_FORMS:
        raise ValueError(f"unknown refinement form {name!r}")
    return _REFINE_FORMS[name]


def _prec_code(name):
    if name not in _PREC_NAMES:
        raise ValueError(f"unknown precision {name!r}")
    return _PREC_NAMES[name]


def _c_params(model):
    """pf_params over the model's host arrays, and the arrays it points into (keep them alive)."""
    arrays = [_dbl_arr(model.h), _dbl_arr(model.mu), _dbl_arr(model.A), _dbl_arr(model.u_noise), _dbl_arr(model.E)]
    nj = None
    if model.n_of_j is not None:
        nj = np.ascontiguousarray(np.asarray(model.n_of_j, dtype=np.int32))
    prm = L.pf_params(h=arrays[0][1], mu=arrays[1][1], A=arrays[2][1], u_noise=arrays[3][1],
                      n_of_j=nj.ctypes.data_as(C.POINTER(C.c_int32)) if nj is not None else None, E=arrays[4][1])
    return prm, (arrays, nj)


def _dbl_arr(x):
    if x is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


class _DevView:
    """Non-owning __cuda_array_interface__ wrapper of a library-owned device array."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


def _copy_device(ptr, n, typestr, torch_dtype):
    if n == 0:
        return torch.empty(0, dtype=torch_dtype, device="cuda")
    t = torch.as_tensor(_DevView(ptr, (n,), typestr), device="cuda")
    return t.clone()


@dataclass
class Model:
    kind: int
    L: int
    N: int = 0
    N_up: int = 0
    N_dn: int = 0
    bc: int = 0
    J: float = 1.0
    Delta: float = 1.0
    t: float = 1.0
    U: float = 0.0
    g0: float = 1.0
    alpha: float = 0.75
    gamma: float = 1.0
    Gamma: float = 1.0
    J2: float = 0.0
    Delta2: float = 1.0
    J3: float = 0.0
    Delta3: float = 1.0
    phi: float = 0.0
    h: object = None
    mu: object = None
    A: object = None
    u_noise: object = None
    n_of_j: object = None
    E: object = None

    @staticmethod
    def from_params(p):
        """From a parameter record with the attribute names of pf_inputs.workloads."""
        k = p.kind
        if k == L.PF_MODEL_XXZ:
            return Model(kind=k, L=p.L, N=p.N, bc=p.bc, J=p.J, Delta=p.Delta, h=p.h, J2=getattr(p, "J2", 0.0),
                         Delta2=getattr(p, "Delta2", 1.0), J3=getattr(p, "J3", 0.0), Delta3=getattr(p, "Delta3", 1.0),
                         phi=getattr(p, "phi", 0.0))
        if k == L.PF_MODEL_QSUN:
            return Model(kind=k, L=p.L, N=p.N, g0=p.g0, alpha=p.alpha, gamma=p.gamma, h=p.h, A=p.A,
                         u_noise=p.u_noise, n_of_j=p.n_of_j)
        if k == L.PF_MODEL_HUBBARD:
            return Model(kind=k, L=p.L, N_up=p.N_up, N_dn=p.N_dn, bc=p.bc, t=p.t, U=p.U, mu=p.mu)
        if k == L.PF_MODEL_QREM:
            return Model(kind=k, L=p.L, Gamma=p.Gamma, E=p.E)
        if k == L.PF_MODEL_QSUN_U1:
            return Model(kind=k, L=p.L, N=p.N, N_up=p.M, g0=p.g0, alpha=p.alpha, gamma=p.gamma, h=p.h, A=p.A,
                         u_noise=p.u_noise, n_of_j=p.n_of_j)
        raise ValueError(f"unknown model kind {k}")

    def c_model(self):
        return L.pf_model(kind=self.kind, L=self.L, N=self.N, N_up=self.N_up, N_dn=self.N_dn, bc=self.bc,
                          J=self.J, Delta=self.Delta, t=self.t, U=self.U, g0=self.g0, alpha=self.alpha,
                          gamma=self.gamma, Gamma=self.Gamma, J2=self.J2, Delta2=self.Delta2, J3=self.J3,
                          Delta3=self.Delta3, phi=self.phi)


class Basis:
    def __init__(self, model, stream=None):
        _install_torch_allocator()
        self.model = model
        h = C.c_void_p()
        check(lib().pf_build_basis(C.byref(model.c_model()), C.byref(h), _stream(stream)), "pf_build_basis")
        self.handle = h
        D, Du, Dd = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().pf_basis_info(h, C.byref(D), C.byref(Du), C.byref(Dd)), "pf_basis_info")
        self.D, self.D_up, self.D_dn = D.value, Du.value, Dd.value

    def states(self):
        """Copy of the state table (XXZ: [D]; Hubbard: up table then down table) as int64."""
        p = C.c_void_p()
        check(lib().pf_basis_states(self.handle, C.byref(p)), "pf_basis_states")
        n = self.D if self.model.kind == L.PF_MODEL_XXZ else (self.D_up + self.D_dn
                                                              if self.model.kind == L.PF_MODEL_HUBBARD else 0)
        if not p.value:
            return torch.empty(0, dtype=torch.int64, device="cuda")
        return _copy_device(p.value, n, "<u4", torch.int32).to(torch.int64) & 0xFFFFFFFF

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                lib().pf_free_basis(self.handle)
                self.handle = None
        except Exception:
            pass


@dataclass
class SolveResult:
    evals: np.ndarray
    resid: np.ndarray
    evecs: torch.Tensor
    report: dict
    status: int


class Hamiltonian:
    """CSR Hamiltonian on the device (FP64) with its rescaled copies H~ (FP64, FP32)."""

    def __init__(self, model, stream=None):
        _install_torch_allocator()
        self.model = model
        self.basis = Basis(model, stream)
        prm, self._keep = _c_params(model)
        h = C.c_void_p()
        check(lib().pf_build_hamiltonian(self.basis.handle, C.byref(model.c_model()), C.byref(prm), C.byref(h),
                                         _stream(stream)), "pf_build_hamiltonian")
        self.handle = h
        D, nnz, nrm = C.c_int64(), C.c_int64(), C.c_double()
        check(lib().pf_ham_info(h, C.byref(D), C.byref(nnz), C.byref(nrm)), "pf_ham_info")
        self.D, self.nnz = D.value, nnz.value

    @staticmethod
    def from_params(p, stream=None):
        return Hamiltonian(Model.from_params(p), stream)

    def __del__(self):
        try:
            if getattr(self, "handle", None):
                lib().pf_free_ham(self.handle)
                self.handle = None
        except Exception:
            pass

    # ---- structure and values
    def csr(self):
        rp, col, val = C.c_void_p(), C.c_void_p(), C.c_void_p()
        check(lib().pf_ham_csr(self.handle, C.byref(rp), C.byref(col), C.byref(val)), "pf_ham_csr")
        torch.cuda.current_stream().synchronize()
        return (_copy_device(rp.value, self.D + 1, "<i8", torch.int64),
                _copy_device(col.value, self.nnz, "<i4", torch.int32),
                _copy_device(val.value, self.nnz, "<f8", torch.float64))

    def set_mapping(self, mapping):
        """How the steps read H~: "csr" or "structured" (QREM only, its default)."""
        m = {"csr": L.PF_MAP_CSR, "structured": L.PF_MAP_STRUCTURED}[mapping]
        check(lib().pf_ham_set_mapping(self.handle, m), "pf_ham_set_mapping")

    def rescaled(self):
        Ec, dE, v64, v32 = C.c_double(), C.c_double(), C.c_void_p(), C.c_void_p()
        check(lib().pf_ham_rescaled(self.handle, C.byref(Ec), C.byref(dE), C.byref(v64), C.byref(v32)),
              "pf_ham_rescaled")
        torch.cuda.current_stream().synchronize()
        return (Ec.value, dE.value, _copy_device(v64.value, self.nnz, "<f8", torch.float64),
                _copy_device(v32.value, self.nnz, "<f4", torch.float32))

    def norm(self):
        D, nnz, nrm = C.c_int64(), C.c_int64(), C.c_double()
        check(lib().pf_ham_info(self.handle, C.byref(D), C.byref(nnz), C.byref(nrm)), "pf_ham_info")
        return nrm.value

    # ---- bounds, rescaling, moments, K
    def spectral_bounds(self, tol=1e-10, stream=None):
        a, b, ra, rb = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        check(lib().pf_spectral_bounds(self.handle, tol, C.byref(a), C.byref(b), C.byref(ra), C.byref(rb),
                                       _stream(stream)), "pf_spectral_bounds")
        return a.value, b.value, ra.value, rb.value

    def set_rescale(self, Ec, dE, stream=None):
        check(lib().pf_set_rescale(self.handle, float(Ec), float(dE), _stream(stream)), "pf_set_rescale")

    def moments(self, stream=None):
        mu, G = C.c_double(), C.c_double()
        check(lib().pf_ham_moments(self.handle, C.byref(mu), C.byref(G), _stream(stream)), "pf_ham_moments")
        return mu.value, G.value

    def choose_K(self, eps, nev, stream=None):
        K = C.c_int32()
        check(lib().pf_choose_K(self.handle, float(eps), int(nev), C.byref(K), _stream(stream)), "pf_choose_K")
        return K.value

    # ---- density of states (kernel polynomial method)
    def kpm_moments(self, N=128, R=32, seed=7, stream=None):
        """mu_n = Tr T_n(H~), n < N, estimated with R random vectors (pf_kpm_moments)."""
        mu = np.zeros(N)
        check(lib().pf_kpm_moments(self.handle, int(N), int(R), C.c_uint64(seed),
                                   mu.ctypes.data_as(C.POINTER(C.c_double)), _stream(stream)), "pf_kpm_moments")
        return mu

    def autotune_block(self, nev, precision="f32", stream=None):
        """(block width, {s: measured step us}, {s: predicted Lanczos filter cost}) from the autotuner."""
        b = C.c_int32()
        us, cost = (C.c_double * 4)(), (C.c_double * 4)()
        check(lib().pf_autotune_block(self.handle, L.PF_F64 if precision == "f64" else L.PF_F32, int(nev),
                                      C.byref(b), us, cost, _stream(stream)), "pf_autotune_block")
        cands = (8, 16, 32, 64)
        return b.value, {c: us[i] for i, c in enumerate(cands)}, {c: cost[i] for i, c in enumerate(cands) if cost[i] > 0}

    def target_abs(self, lam_t):
        """Absolute energy of a rescaled target E~ (for solve(target_abs=...))."""
        Ec, dE, _, _ = self.rescaled()
        return Ec + dE * float(lam_t)

    # ---- kernels
    def clenshaw_step(self, V, B1, B2, out, a, alpha, beta, use_H=False, stream=None):
        prec = _block_prec(V)
        s = V.shape[1]
        check(lib().pf_clenshaw_step(self.handle, prec, s, _ptr(V), _ptr(B1), _ptr(B2), _ptr(out), float(a),
                                     float(alpha), float(beta), int(bool(use_H)), _stream(stream)),
              "pf_clenshaw_step")
        return out

    def filter_apply(self, V, coeffs, W=None, stream=None):
        prec = _block_prec(V)
        W = torch.empty_like(V) if W is None else W
        c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
        check(lib().pf_filter_apply(self.handle, prec, V.shape[1], _ptr(V), _ptr(W),
                                    c.ctypes.data_as(C.POINTER(C.c_double)), len(c) - 1, _stream(stream)),
              "pf_filter_apply")
        return W

    def filter_apply_cols(self, V, coeffs, W=None, stream=None):
        """W[:, j] = P_j(H~) V[:, j] with coeffs[:, j] the Chebyshev coefficients of column j
        ((K+1) x s, pf_filter_apply_cols)."""
        prec = _block_prec(V)
        W = torch.empty_like(V) if W is None else W
        c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
        if c.ndim != 2 or c.shape[1] != V.shape[1]:
            raise ValueError("coeffs must be (K+1) x s")
        check(lib().pf_filter_apply_cols(self.handle, prec, V.shape[1], _ptr(V), _ptr(W),
                                         c.ctypes.data_as(C.POINTER(C.c_double)), c.shape[0] - 1, _stream(stream)),
              "pf_filter_apply_cols")
        return W

    # ---- the solve
    def solve_complex(self, eps, nev, K, block=32, precision="f64", return_vectors=True, target_abs=None, stream=None,
                      raise_on_notconv=True, **opts):
        """The nev eigenpairs of a complex-Hermitian model (phi != 0) nearest the target
        (pf_polfed_solve_complex): evals, resid, and evecs as a (D, nev) complex128 tensor, D the
        sector's dimension (the handle's D is 2 D, the real embedding)."""
        o = _make_opts(block, precision, target_abs, opts)
        evals = np.zeros(nev)
        resid = np.zeros(nev)
        Dc = self.D // 2
        buf = torch.empty((nev, Dc, 2), dtype=torch.float64, device="cuda") if return_vectors else None
        rep = L.pf_report()
        st = lib().pf_polfed_solve_complex(self.handle, float(eps), int(nev), int(K), C.byref(o),
                                           evals.ctypes.data_as(C.POINTER(C.c_double)), _ptr(buf),
                                           resid.ctypes.data_as(C.POINTER(C.c_double)), C.byref(rep), _stream(stream))
        if st not in (L.PF_OK, L.PF_ENOTCONV) or (st == L.PF_ENOTCONV and raise_on_notconv):
            check(st, "pf_polfed_solve_complex")
        evecs = torch.view_as_complex(buf).t() if buf is not None else None
        return SolveResult(evals=evals, resid=resid, evecs=evecs, report=rep.as_dict(), status=st)

    def solve(self, eps, nev, K, block=32, precision="f64", return_vectors=True, target_abs=None, stream=None,
              raise_on_notconv=True, **opts):
        o = _make_opts(block, precision, target_abs, opts)
        evals = np.zeros(nev)
        resid = np.zeros(nev)
        evecs = torch.empty((nev, self.D), dtype=torch.float64, device="cuda") if return_vectors else None
        rep = L.pf_report()
        st = lib().pf_polfed_solve(self.handle, float(eps), int(nev), int(K), C.byref(o),
                                   evals.ctypes.data_as(C.POINTER(C.c_double)), _ptr(evecs),
                                   resid.ctypes.data_as(C.POINTER(C.c_double)), C.byref(rep), _stream(stream))
        if st not in (L.PF_OK, L.PF_ENOTCONV) or (st == L.PF_ENOTCONV and raise_on_notconv):
            check(st, "pf_polfed_solve")
        # evecs buffer is D x nev column-major == (nev, D) row-major; expose as (D, nev)
        return SolveResult(evals=evals, resid=resid, evecs=evecs.t() if evecs is not None else None,
                           report=rep.as_dict(), status=st)


def _make_opts(block, precision, target_abs, opts):
    o = L.pf_solve_opts()
    lib().pf_default_opts(C.byref(o))
    o.block = block
    o.precision = L.PF_F64 if precision == "f64" else L.PF_F32
    for k, v in opts.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        if k in ("refine_precision", "orth_precision") and isinstance(v, str):
            v = _prec_code(v)
        if k == "refine_form" and isinstance(v, str):
            v = _refine_form_code(v)
        setattr(o, k, v)
    if target_abs is not None:
        o.use_abs_target = 1
        o.target_abs = float(target_abs)
    return o


def filter_apply_batch(items, form="auto", stream=None):
    """W_j = P_j(H~_j) V_j for items (H, V, coeffs) of one dtype and block width, together.

    form: "auto" (autotuner), "steps" (one launch per step), "graph" (the steps as a CUDA
    graph) or a cluster size 1/2/4/8/16 (one persistent launch)."""
    _install_torch_allocator()
    n = len(items)
    if n == 0:
        return []
    V0 = items[0][1]
    prec = _block_prec(V0)
    arr = (L.pf_filter_item * n)()
    keep, outs = [], []
    for j, (H, V, coeffs) in enumerate(items):
        c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64))
        W = torch.empty_like(V)
        keep.append(c)
        outs.append(W)
        arr[j].H = H.handle.value if isinstance(H.handle, C.c_void_p) else H.handle
        arr[j].V = V.data_ptr()
        arr[j].W = W.data_ptr()
        arr[j].coeffs = c.ctypes.data_as(C.POINTER(C.c_double))
        arr[j].K = len(c) - 1
    f = {"auto": L.PF_FORM_AUTO, "steps": L.PF_FORM_STEPS, "graph": L.PF_FORM_GRAPH}.get(form, form)
    check(lib().pf_filter_apply_batch(arr, n, prec, V0.shape[1], int(f), _stream(stream)), "pf_filter_apply_batch")
    return outs


def filter_tune(H, K, s=32, precision="f32", n=1, stream=None):
    """The autotuner's form for a group of n items shaped like H: (form, measured per-step us).

    form 0 = per-step sweep (plain recurrence for n = 1), c >= 1 = persistent clusters of c CTAs."""
    _install_torch_allocator()
    f = C.c_int32()
    us = (C.c_double * 8)()
    check(lib().pf_filter_tune(H.handle, _prec_code(precision), int(s), int(K), int(n),
                               C.byref(f), us, _stream(stream)), "pf_filter_tune")
    names = ["raw", "sweep", "sweep_copies", "c1", "c2", "c4", "c8", "c16"]
    return f.value, {k: us[i] for i, k in enumerate(names) if us[i] > 0}


def solve_batch(problems, block=32, precision="f64", return_vectors=False, stream=None, **opts):
    """Solve independent problems together.  problems: dicts with keys H, eps, nev, K and
    optionally target_abs, block, precision (overriding the call's).  Returns one
    SolveResult per problem (status per problem)."""
    n = len(problems)
    arr = (L.pf_solve_item * n)()
    keep = []
    for j, pb in enumerate(problems):
        H, nev = pb["H"], int(pb["nev"])
        o = _make_opts(pb.get("block", block), pb.get("precision", precision), pb.get("target_abs"), opts)
        ev, rs, rep = np.zeros(nev), np.zeros(nev), L.pf_report()
        vec = torch.empty((nev, H.D), dtype=torch.float64, device="cuda") if return_vectors else None
        keep.append((o, ev, rs, rep, vec))
        arr[j].H = H.handle.value if isinstance(H.handle, C.c_void_p) else H.handle
        arr[j].target_eps = float(pb.get("eps", 0.5))
        arr[j].nev = nev
        arr[j].K = int(pb["K"])
        arr[j].opts = C.pointer(o)
        arr[j].evals = ev.ctypes.data_as(C.POINTER(C.c_double))
        arr[j].evecs = vec.data_ptr() if vec is not None else None
        arr[j].resid = rs.ctypes.data_as(C.POINTER(C.c_double))
        arr[j].rep = C.pointer(rep)
    st = lib().pf_polfed_solve_batch(arr, n, _stream(stream))
    if st not in (L.PF_OK, L.PF_ENOTCONV, L.PF_EINVAL, L.PF_ESTATE, L.PF_EBREAKDOWN):
        check(st, "pf_polfed_solve_batch")
    out = []
    for j, (o, ev, rs, rep, vec) in enumerate(keep):
        out.append(SolveResult(evals=ev, resid=rs, evecs=vec.t() if vec is not None else None,
                               report=rep.as_dict(), status=arr[j].status))
    return out


def solve_footprint(D, nnz, nev, block=32, precision="f64"):
    """Device bytes one solve holds at its peak (the server's admission measure)."""
    b = C.c_int64()
    check(lib().pf_solve_footprint(int(D), int(nnz), int(nev), int(block),
                                   L.PF_F64 if precision == "f64" else L.PF_F32, C.byref(b)), "pf_solve_footprint")
    return b.value


@dataclass
class RequestResult:
    id: int
    status: int
    evals: np.ndarray
    resid: np.ndarray
    report: dict
    latency_ms: float
    queue_ms: float
    footprint_bytes: int


class Server:
    """Continuous-batching solve server (pf_server_*): submit requests, step, take results."""

    def __init__(self, block=32, precision="f32", max_active=64, mem_budget_bytes=0, res_tol=0.0, bounds_tol=0.0,
                 seed=0, stream=None, refine_precision="f64", refine_form="default"):
        _install_torch_allocator()
        cfg = L.pf_server_config(block=block, precision=L.PF_F64 if precision == "f64" else L.PF_F32,
                                 max_active=max_active, mem_budget_bytes=int(mem_budget_bytes), res_tol=res_tol,
                                 bounds_tol=bounds_tol, seed=seed, refine_precision=_prec_code(refine_precision),
                                 refine_form=_refine_form_code(refine_form))
        self._stream = stream
        h = C.c_void_p()
        check(lib().pf_server_create(C.byref(cfg), _stream(stream), C.byref(h)), "pf_server_create")
        self.handle = h
        self._nev = {}

    def submit(self, model, eps, nev):
        prm, keep = _c_params(model)
        rid = C.c_int64()
        check(lib().pf_server_submit(self.handle, C.byref(model.c_model()), C.byref(prm), float(eps), int(nev),
                                     C.byref(rid)), "pf_server_submit")
        self._nev[rid.value] = int(nev)
        return rid.value

    def step(self):
        q, a, f = C.c_int32(), C.c_int32(), C.c_int32()
        check(lib().pf_server_step(self.handle, C.byref(q), C.byref(a), C.byref(f)), "pf_server_step")
        return q.value, a.value, f.value

    def take(self, rid):
        """The finished request's result, or None while it is queued or resident."""
        nev = self._nev[rid]
        ev, rs, rep, info = np.zeros(nev), np.zeros(nev), L.pf_report(), L.pf_request_info()
        st = lib().pf_server_take(self.handle, int(rid), ev.ctypes.data_as(C.POINTER(C.c_double)),
                                  rs.ctypes.data_as(C.POINTER(C.c_double)), C.byref(rep), C.byref(info))
        if st == L.PF_ESTATE:
            return None
        check(st, "pf_server_take")
        del self._nev[rid]
        return RequestResult(id=rid, status=info.status, evals=ev, resid=rs, report=rep.as_dict(),
                             latency_ms=info.latency_ms, queue_ms=info.queue_ms,
                             footprint_bytes=info.footprint_bytes)

    def memory(self):
        u, b = C.c_int64(), C.c_int64()
        check(lib().pf_server_memory(self.handle, C.byref(u), C.byref(b)), "pf_server_memory")
        return u.value, b.value

    def close(self):
        if getattr(self, "handle", None):
            lib().pf_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kpm_dos(mu, x):
    """rho_KPM at the points x (Jackson kernel)."""
    m = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    xs = np.ascontiguousarray(np.atleast_1d(np.asarray(x, dtype=np.float64)))
    out = np.zeros_like(xs)
    check(lib().pf_kpm_dos(m.ctypes.data_as(C.POINTER(C.c_double)), len(m), xs.ctypes.data_as(C.POINTER(C.c_double)),
                           len(xs), out.ctypes.data_as(C.POINTER(C.c_double))), "pf_kpm_dos")
    return out


def kpm_target(mu, eta=0.0):
    """Rescaled target E~: :maxdos for eta = 0, (:offset, eta) otherwise."""
    m = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    t = C.c_double()
    check(lib().pf_kpm_target(m.ctypes.data_as(C.POINTER(C.c_double)), len(m), float(eta), C.byref(t)),
          "pf_kpm_target")
    return t.value


def choose_K_kpm(mu, lam_t, nev):
    """K from Eq. condition_for_K with the KPM density at lam_t."""
    m = np.ascontiguousarray(np.asarray(mu, dtype=np.float64))
    K = C.c_int32()
    check(lib().pf_choose_K_kpm(m.ctypes.data_as(C.POINTER(C.c_double)), len(m), float(lam_t), int(nev), C.byref(K)),
          "pf_choose_K_kpm")
    return K.value


def filter_coefficients(lam_t, K, stream=None):
    _install_torch_allocator()
    c = np.zeros(K + 1)
    check(lib().pf_filter_coefficients(float(lam_t), int(K), c.ctypes.data_as(C.POINTER(C.c_double)),
                                       _stream(stream)), "pf_filter_coefficients")
    return c


def sym_eig_select(A, idx, stream=None):
    """Eigenpairs of the symmetric n x n device matrix A (FP64) for the ascending-order indices idx
    (pf_sym_eig_select, the H_L eigensolver): returns (w ndarray [q], Z tensor n x q)."""
    n = A.shape[0]
    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 2 or A.shape[1] != n:
        raise ValueError("A must be a square float64 CUDA tensor")
    A = A.contiguous()
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    q = len(ix)
    w = np.zeros(q)
    Z = torch.empty((q, n), dtype=torch.float64, device="cuda")     # column k of the n x q result = row k
    check(lib().pf_sym_eig_select(_ptr(A), n, n, ix.ctypes.data_as(C.POINTER(C.c_int32)), q,
                                  w.ctypes.data_as(C.POINTER(C.c_double)), _ptr(Z), n, _stream(stream)),
          "pf_sym_eig_select")
    return w, Z.t()


def start_block(D, s, seed, stream=None):
    out = torch.empty((D, s), dtype=torch.float64, device="cuda")
    check(lib().pf_start_block(int(D), int(s), C.c_uint64(seed), _ptr(out), _stream(stream)), "pf_start_block")
    return out
