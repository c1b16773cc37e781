"""B300-native POLFED hot path: basis/CSR builders, fused Clenshaw-SpMM filter and block
Lanczos on the device, behind the C ABI of include/polfed.h."""
from .api import Model, Basis, Hamiltonian, SolveResult, filter_coefficients, start_block  # noqa: F401
from ._lib import lib, LIB_PATH, PolfedError  # noqa: F401
