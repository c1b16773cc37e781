"""B300-native POLFED hot path: basis/CSR builders, fused Clenshaw-SpMM filter and block
Lanczos on the device, behind the C ABI of include/polfed.h."""
from .api import (Model, Basis, Hamiltonian, SolveResult, RequestResult, Server, filter_coefficients,  # noqa: F401
                  filter_apply_batch, filter_tune, solve_batch, kpm_dos, kpm_target, choose_K_kpm, solve_footprint, start_block,
                  sym_eig_select)
from ._lib import lib, LIB_PATH, PolfedError  # noqa: F401
