"""ctypes declarations of the C ABI in include/polfed.h (argument marshalling only).

Loading fails loudly when libpolfed.so is missing: there is no CPU fallback.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpolfed.so")

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ENOTCONV, PF_ETIMEOUT, PF_ECUDA, PF_ESTATE, PF_EBREAKDOWN = range(8)
PF_MODEL_XXZ, PF_MODEL_QSUN, PF_MODEL_HUBBARD, PF_MODEL_QREM, PF_MODEL_QSUN_U1 = 0, 1, 2, 3, 4
PF_MAP_CSR, PF_MAP_STRUCTURED = 0, 1
PF_F64, PF_F32, PF_DF64 = 0, 1, 2
PF_REFINE_DIRECT, PF_REFINE_CORRECTION = 1, 2
PF_FORM_AUTO, PF_FORM_STEPS, PF_FORM_GRAPH = -1, 0, -2


class pf_model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("L", C.c_int32), ("N", C.c_int32), ("N_up", C.c_int32),
                ("N_dn", C.c_int32), ("bc", C.c_int32), ("J", C.c_double), ("Delta", C.c_double),
                ("t", C.c_double), ("U", C.c_double), ("g0", C.c_double), ("alpha", C.c_double),
                ("gamma", C.c_double), ("Gamma", C.c_double), ("J2", C.c_double), ("Delta2", C.c_double),
                ("J3", C.c_double), ("Delta3", C.c_double), ("phi", C.c_double)]


class pf_params(C.Structure):
    _fields_ = [("h", C.POINTER(C.c_double)), ("mu", C.POINTER(C.c_double)), ("A", C.POINTER(C.c_double)),
                ("u_noise", C.POINTER(C.c_double)), ("n_of_j", C.POINTER(C.c_int32)),
                ("E", C.POINTER(C.c_double))]


class pf_solve_opts(C.Structure):
    _fields_ = [("block", C.c_int32), ("precision", C.c_int32), ("nev_guard", C.c_int32),
                ("check_first", C.c_int32), ("check_every", C.c_int32), ("max_blocks", C.c_int32),
                ("eta", C.c_double), ("tol", C.c_double), ("tol_f32", C.c_double), ("res_tol", C.c_double),
                ("refine_passes", C.c_int32), ("refine_K", C.c_int32), ("seed", C.c_uint64),
                ("use_abs_target", C.c_int32), ("target_abs", C.c_double), ("refine_shift", C.c_double),
                ("refine_reserve", C.c_int32), ("refine_full_set", C.c_int32), ("refine_guard_lock", C.c_double),
                ("refine_lock", C.c_double), ("refine_precision", C.c_int32), ("refine_form", C.c_int32),
                ("orth_precision", C.c_int32)]


class pf_report(C.Structure):
    _fields_ = [("status", C.c_int32), ("K", C.c_int32), ("blocks", C.c_int32), ("krylov_dim", C.c_int32),
                ("nev_guard", C.c_int32), ("converged", C.c_int32), ("checks", C.c_int32),
                ("refine_passes", C.c_int32), ("filter_steps_f32", C.c_int64), ("filter_steps_f64", C.c_int64),
                ("emin", C.c_double), ("emax", C.c_double), ("Ec", C.c_double), ("dE", C.c_double),
                ("lambda_", C.c_double), ("lambda_t", C.c_double), ("hnorm", C.c_double),
                ("max_residual", C.c_double), ("ms_filter_f32", C.c_double), ("ms_filter_f64", C.c_double),
                ("ms_orth", C.c_double), ("ms_qr", C.c_double), ("ms_check", C.c_double),
                ("ms_extract", C.c_double), ("ms_refine", C.c_double), ("ms_total", C.c_double),
                ("max_residual_unrefined", C.c_double), ("refine_active", C.c_int32 * 8),
                ("refine_residual", C.c_double * 8)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if not isinstance(v, (int, float)) else v
        return out


class pf_filter_item(C.Structure):
    _fields_ = [("H", C.c_void_p), ("V", C.c_void_p), ("W", C.c_void_p), ("coeffs", C.POINTER(C.c_double)),
                ("K", C.c_int32)]


class pf_solve_item(C.Structure):
    _fields_ = [("H", C.c_void_p), ("target_eps", C.c_double), ("nev", C.c_int32), ("K", C.c_int32),
                ("opts", C.POINTER(pf_solve_opts)), ("evals", C.POINTER(C.c_double)), ("evecs", C.c_void_p),
                ("resid", C.POINTER(C.c_double)), ("rep", C.POINTER(pf_report)), ("status", C.c_int32)]


class pf_server_config(C.Structure):
    _fields_ = [("block", C.c_int32), ("precision", C.c_int32), ("max_active", C.c_int32),
                ("mem_budget_bytes", C.c_int64), ("res_tol", C.c_double), ("bounds_tol", C.c_double),
                ("seed", C.c_uint64), ("refine_precision", C.c_int32), ("refine_form", C.c_int32)]


class pf_request_info(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("nev", C.c_int32), ("footprint_bytes", C.c_int64),
                ("queue_ms", C.c_double), ("latency_ms", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

vp, i32, i64, dbl, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
P = C.POINTER

# name -> (restype, argtypes); every function declared in include/polfed.h
PROTOTYPES = {
    "pf_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
    "pf_status_str": (C.c_char_p, [i32]),
    "pf_last_cuda_error": (C.c_char_p, []),
    "pf_kernel_launches": (C.c_longlong, []),
    "pf_build_basis": (i32, [P(pf_model), P(vp), vp]),
    "pf_basis_info": (i32, [vp, P(i64), P(i64), P(i64)]),
    "pf_basis_states": (i32, [vp, P(vp)]),
    "pf_free_basis": (None, [vp]),
    "pf_build_hamiltonian": (i32, [vp, P(pf_model), P(pf_params), P(vp), vp]),
    "pf_ham_info": (i32, [vp, P(i64), P(i64), P(dbl)]),
    "pf_ham_csr": (i32, [vp, P(vp), P(vp), P(vp)]),
    "pf_free_ham": (None, [vp]),
    "pf_spectral_bounds": (i32, [vp, dbl, P(dbl), P(dbl), P(dbl), P(dbl), vp]),
    "pf_set_rescale": (i32, [vp, dbl, dbl, vp]),
    "pf_ham_rescaled": (i32, [vp, P(dbl), P(dbl), P(vp), P(vp)]),
    "pf_ham_set_mapping": (i32, [vp, i32]),
    "pf_ham_moments": (i32, [vp, P(dbl), P(dbl), vp]),
    "pf_filter_coefficients": (i32, [dbl, i32, P(dbl), vp]),
    "pf_choose_K": (i32, [vp, dbl, i32, P(i32), vp]),
    "pf_clenshaw_step": (i32, [vp, i32, i32, vp, vp, vp, vp, dbl, dbl, dbl, i32, vp]),
    "pf_filter_apply": (i32, [vp, i32, i32, vp, vp, P(dbl), i32, vp]),
    "pf_filter_apply_cols": (i32, [vp, i32, i32, vp, vp, P(dbl), i32, vp]),
    "pf_filter_apply_noalloc": (i32, [vp, i32, i32, vp, vp, P(dbl), i32, vp]),
    "pf_default_opts": (None, [P(pf_solve_opts)]),
    "pf_polfed_solve": (i32, [vp, dbl, i32, i32, P(pf_solve_opts), P(dbl), vp, P(dbl), P(pf_report), vp]),
    "pf_polfed_solve_complex": (i32, [vp, dbl, i32, i32, P(pf_solve_opts), P(dbl), vp, P(dbl), P(pf_report), vp]),
    "pf_start_block": (i32, [i64, i32, u64, vp, vp]),
    "pf_sym_eig_select": (i32, [vp, i32, i32, P(i32), i32, P(dbl), vp, i32, vp]),
    "pf_filter_apply_batch": (i32, [P(pf_filter_item), i32, i32, i32, i32, vp]),
    "pf_filter_tune": (i32, [vp, i32, i32, i32, i32, P(i32), P(dbl), vp]),
    "pf_polfed_solve_batch": (i32, [P(pf_solve_item), i32, vp]),
    "pf_solve_footprint": (i32, [i64, i64, i32, i32, i32, P(i64)]),
    "pf_server_create": (i32, [P(pf_server_config), vp, P(vp)]),
    "pf_server_submit": (i32, [vp, P(pf_model), P(pf_params), dbl, i32, P(i64)]),
    "pf_server_step": (i32, [vp, P(i32), P(i32), P(i32)]),
    "pf_server_take": (i32, [vp, i64, P(dbl), P(dbl), P(pf_report), P(pf_request_info)]),
    "pf_server_memory": (i32, [vp, P(i64), P(i64)]),
    "pf_server_destroy": (None, [vp]),
    "pf_kpm_moments": (i32, [vp, i32, i32, u64, P(dbl), vp]),
    "pf_kpm_dos": (i32, [P(dbl), i32, P(dbl), i32, P(dbl)]),
    "pf_kpm_target": (i32, [P(dbl), i32, dbl, P(dbl)]),
    "pf_choose_K_kpm": (i32, [P(dbl), i32, dbl, i32, P(i32)]),
    "pf_autotune_block": (i32, [vp, i32, i32, P(i32), P(dbl), P(dbl), vp]),
}

_lib = None


def lib():
    """The loaded library; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpolfed.so not found at {LIB_PATH}; build it first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PolfedError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().pf_status_str(status).decode()
        if status == PF_ECUDA:
            msg += " (" + lib().pf_last_cuda_error().decode() + ")"
        super().__init__(f"{where}: {msg}")
        self.status = status


def check(status, where):
    if status != PF_OK:
        raise PolfedError(status, where)
