/*
 * polfed.h -- C ABI of the B300 (sm_103a) POLFED hot path.
 *
 * POLFED computes the eigenpairs of a sparse real-symmetric Hamiltonian H that lie
 * nearest a target energy lambda by running block Lanczos on the polynomial filter
 * P(H~) = (1/chi) sum_{n=0..K} c_n T_n(H~) (paper, Sec. 3.2, Eq. transformation and
 * Eq. transformationCoefficients), applied on the fly with the Clenshaw recurrence
 * (Sec. 4.4, Eq. clenshaw_chebyshev_prod).  H~ = (H - E_c)/dE is H rescaled into
 * [-1, 1] (Eq. rescaledMatrix).
 *
 * Conventions for every entry point:
 *  - Return value: a pf_status.  No call aborts, traps or throws across this ABI.
 *  - Pointers documented "device" must be CUDA device memory of the current device;
 *    "host" pointers are ordinary host memory.  The caller owns every buffer it
 *    passes in; the library never frees caller memory.
 *  - Handles (pf_basis, pf_ham) are owned by the library and released with
 *    pf_free_basis / pf_free_ham.  Their device memory comes from the allocator
 *    installed by pf_set_allocator (default: cudaMallocAsync / cudaFreeAsync).
 *  - Work is enqueued on the given stream.  Calls that return host scalars
 *    synchronise that stream before returning.  A handle must not be used by two
 *    threads at once; distinct handles are independent: the library's process-wide
 *    state (tuning caches, stream pools, kernel attributes) is guarded by locks or set
 *    once, and kernel shared-memory limits are only ever raised.
 *  - Vector blocks are D x s, row-major (the s entries of a row are contiguous).
 */
#ifndef POLFED_H
#define POLFED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* pf_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  PF_OK = 0,
  PF_EINVAL = 1,    /* bad argument: shape, nev > D, K < 1, eps outside [0,1], ...  */
  PF_ENOMEM = 2,    /* the allocator returned NULL                                    */
  PF_ENOTCONV = 3,  /* not converged within the Krylov budget; outputs hold the best
                       pairs found, with their residuals                              */
  PF_ETIMEOUT = 4,  /* a device-side wait reached its iteration limit                 */
  PF_ECUDA = 5,     /* a CUDA call failed; pf_last_cuda_error() names it              */
  PF_ESTATE = 6,    /* call order violated (e.g. solve before pf_spectral_bounds)     */
  PF_EBREAKDOWN = 7 /* Cholesky-QR breakdown the recovery path could not repair       */
} pf_status;

typedef enum {
  PF_MODEL_XXZ = 0, PF_MODEL_QSUN = 1, PF_MODEL_HUBBARD = 2, PF_MODEL_QREM = 3, PF_MODEL_QSUN_U1 = 4
} pf_model_kind;
typedef enum { PF_BC_PERIODIC = 0, PF_BC_OPEN = 1 } pf_boundary;
/* Arithmetic of a filter (Clenshaw) step.
 *  PF_F64   double blocks, FP64 values and arithmetic.
 *  PF_F32   float blocks, FP32 values and arithmetic.
 *  PF_DF64  pair-float ("double-float", Dekker 1971): every entry is a pair of floats
 *           (hi, lo), value hi + lo, stored interleaved (8 bytes per entry, a D x s block
 *           is D x s x 2 floats, row-major); products are split exactly with FMA and sums
 *           carried with Knuth's two-sum, so a step's relative rounding error is about
 *           2^-47 (FP64 gives 2^-53) while it runs on the FP32 units.  The exponent
 *           range is FP32's (|x| < 3.4e38): a recurrence on a spectrum inside [-1, 1]
 *           stays within (K + 1) max|a_n| times the input's size.                  */
typedef enum { PF_F64 = 0, PF_F32 = 1, PF_DF64 = 2 } pf_precision;

/* Model description (paper App. A).
 *  XXZ (Eq. xxz): L sites, N up spins (S^z_tot sector), couplings J, Delta, fields h_i.
 *     Bit i of a basis state is 1 when spin i is up; basis = L-bit integers with
 *     popcount N in ascending order; row = rank in that order.  J2, Delta2 and J3,
 *     Delta3 add the bonds (i, i+2) and (i, i+3) of the J1-J2 (Eq. j1j2) and
 *     J1-J2-J3 (Eq. j1j2j3) chains; a zero coupling adds no bonds.
 *  Quantum sun (Eq. qsun): N dot spins in the top N bits, L outer spins in bits
 *     0..L-1; D = 2^(N+L), row = state.  H_dot = gamma (A + A^T)/sqrt(2)/sqrt(2^N+1);
 *     ray j couples dot spin n(j) and outer spin j with g0 alpha^(j + u_noise_j)/4.
 *  Fermi-Hubbard (not in the paper): L sites, N_up / N_dn fermions, hopping t,
 *     interaction U, potentials mu_i; row = rank_up * D_dn + rank_dn; Jordan-Wigner
 *     order: all up modes, then all down modes.
 *  U(1) quantum sun (Eq. qsun:U1): the quantum sun's N dot and L outer spins in the
 *     sector of N_up up spins among N + L (rows as for XXZ over N + L bits); the dot
 *     matrix keeps only popcount-conserving elements and is normalised on the sector
 *     (Tr(H_dot^2)/D = gamma^2); rays S^x S^x + S^y S^y flip antiparallel pairs with
 *     g0 alpha^u_j / 2.
 *  QREM (Eq. qrem): L spins, full space D = 2^L, row = state; diagonal E_alpha,
 *     single spin flips alpha -> alpha ^ (1 << i) with element -Gamma.              */
typedef struct {
  int32_t kind;     /* pf_model_kind                                   */
  int32_t L;        /* sites (XXZ, Hubbard) or outer spins (quantum sun) */
  int32_t N;        /* XXZ: up spins; quantum sun: dot spins            */
  int32_t N_up, N_dn;
  int32_t bc;       /* pf_boundary (XXZ, Hubbard)                       */
  double J, Delta;  /* XXZ                                              */
  double t, U;      /* Hubbard                                          */
  double g0, alpha, gamma; /* quantum sun                               */
  double Gamma;     /* QREM transverse field                            */
  double J2, Delta2;  /* XXZ: next-nearest couplings, Eq. j1j2 (J2 = 0: none)   */
  double J3, Delta3;  /* XXZ: third-neighbour couplings, Eq. j1j2j3 (J3 = 0: none) */
  double phi;         /* XXZ: flux per bond; != 0 makes H complex Hermitian (needs
                         J2 = J3 = 0 and L >= 3), see below                           */
} pf_model;

/* Complex-Hermitian ring (Sec. 2 allows complex-Hermitian H): with phi != 0 the XXZ hop of
 * bond (i, j) is (J/2) e^{+i phi} S+_i S-_j + h.c. (element (J*0.5) cos(phi) +- i (J*0.5) sin(phi),
 * + when the row's state has spin i up and j down; cos and sin from the host C library).  The
 * Hamiltonian handle then holds the real symmetric embedding [[A, -B], [B, A]] of H = A + iB, of
 * dimension 2 D (D the sector's states; pf_ham_info reports 2 D): row r < D carries A[r,c] at
 * column c and -B[r,c] at D + c, row D + r carries B[r,c] at c and A[r,c] at D + c, exact zeros
 * omitted except the diagonal.  Its spectrum is H's with every eigenvalue twice and [x; y] is an
 * eigenvector exactly when x + iy is one of H, so every real entry point (bounds, K, filters,
 * pf_polfed_solve) works on it unchanged; pf_polfed_solve_complex returns H's own eigenpairs.   */

/* Disorder and random couplings, host arrays (copied during the call).          */
typedef struct {
  const double* h;        /* XXZ and quantum-sun fields, [L]                        */
  const double* mu;       /* Hubbard on-site potentials, [L]                        */
  const double* A;        /* quantum-sun raw normals, [2^N * 2^N] row-major         */
  const double* u_noise;  /* quantum-sun exponent noise u_j - j, [L]                */
  const int32_t* n_of_j;  /* quantum-sun dot spin coupled to outer spin j, [L]      */
  const double* E;        /* QREM energies E_alpha, [2^L]                           */
} pf_params;

typedef struct pf_basis pf_basis;
typedef struct pf_ham pf_ham;

/* Device-memory hook.  alloc(ctx, bytes, stream) returns device memory or NULL;
 * release(ctx, ptr, stream) returns it.  Passing NULL for both restores the
 * default (cudaMallocAsync / cudaFreeAsync on the call's stream).             */
typedef void* (*pf_alloc_fn)(void* ctx, size_t bytes, pf_stream_t stream);
typedef void (*pf_free_fn)(void* ctx, void* ptr, pf_stream_t stream);
pf_status pf_set_allocator(pf_alloc_fn alloc, pf_free_fn release, void* ctx);

const char* pf_status_str(pf_status s);
const char* pf_last_cuda_error(void);   /* thread-local text of the last CUDA failure */
/* Cumulative number of kernels this library has launched in the process (diagnostic). */
long long pf_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * (a1) Basis enumeration.  Sec. 2 intro / App. A.2: the S^z sector of L spins with
 * N up has dimension binom(L, N).  Unranking uses the combinatorial number system.
 *   m   : host, model description.
 *   out : receives a new handle.
 * Errors: PF_EINVAL for L outside [1, 32] (XXZ/Hubbard; N+L <= 30 for the quantum
 * sun), N outside [0, L]; PF_ENOMEM; PF_ECUDA.                                  */
pf_status pf_build_basis(const pf_model* m, pf_basis** out, pf_stream_t stream);
/* D; for Hubbard also the up/down table lengths (else 0).  Synchronises.        */
pf_status pf_basis_info(const pf_basis* b, int64_t* D, int64_t* D_up, int64_t* D_dn);
/* Device pointer to the state table: XXZ states[D]; Hubbard up[D_up] followed by
 * dn[D_dn]; quantum sun: NULL (row = state).  Owned by the handle.             */
pf_status pf_basis_states(const pf_basis* b, const uint32_t** states);
void pf_free_basis(pf_basis* b);

/* ---------------------------------------------------------------------------
 * (a2) Hamiltonian construction: CSR of H (count pass, scan, fill), FP64 values.
 * Eq. xxz, Eq. qsun, Hubbard as above.  Columns ascending in each row; diagonal
 * always stored; repeated (row, col) terms summed in generation order.  Diagonal
 * values are summed term by term without fused multiply-add, so they agree bit for
 * bit with a plain left-to-right FP64 sum.
 *   b, m : the basis built from the same model; p: host disorder arrays.
 * Errors: PF_EINVAL (model/basis mismatch, missing arrays); PF_ENOMEM; PF_ECUDA.   */
pf_status pf_build_hamiltonian(const pf_basis* b, const pf_model* m, const pf_params* p,
                               pf_ham** out, pf_stream_t stream);
/* D, nnz, and ||H|| = max(|Emin|, |Emax|) once pf_spectral_bounds ran (else 0).  */
pf_status pf_ham_info(const pf_ham* H, int64_t* D, int64_t* nnz, double* norm_est);
/* Device CSR arrays (row_ptr int64[D+1], col int32[nnz], val float64[nnz]) of H. */
pf_status pf_ham_csr(const pf_ham* H, const int64_t** row_ptr, const int32_t** col,
                     const double** val);
void pf_free_ham(pf_ham* H);

/* ---------------------------------------------------------------------------
 * (a3) Spectral bounds by FP64 block Lanczos on H (Sec. 2.1-2.2, Eq. lan_criterion),
 * stopping when both extreme Ritz pairs have residual <= tol * max|theta|.  Then
 * sets the rescaling (Eq. rescaledMatrix) on the handle, over the interval padded
 * by the residuals and 1e-3 of the half-width, and writes H~ in FP64 and FP32.
 *   tol <= 0 selects 1e-10.  emin/emax/rmin/rmax: host outputs (rmin/rmax may be NULL).
 * Synchronises.  Errors: PF_ENOTCONV, PF_ENOMEM, PF_ECUDA.                         */
pf_status pf_spectral_bounds(pf_ham* H, double tol, double* emin, double* emax, double* rmin,
                             double* rmax, pf_stream_t stream);
/* Set the rescaling directly (E_c, dE) and write H~ values; for tests and for callers
 * that know their bounds.                                                          */
pf_status pf_set_rescale(pf_ham* H, double Ec, double dE, pf_stream_t stream);
/* How the Clenshaw steps read H~ (custom mappings, Sec. 5.7-5.8).
 *  PF_MAP_CSR         the stored CSR arrays (every model; the default except QREM).
 *  PF_MAP_STRUCTURED  QREM (its default): a row's columns r ^ (1 << i) are generated in
 *                     registers in ascending order and every off-diagonal element is the one
 *                     value -Gamma / dE; only the diagonal is read.  Nearest-neighbour XXZ
 *                     (J2 = J3 = 0, L >= 3; its default): FP32 steps read the CSR columns with
 *                     the one off-diagonal value (J/2) / dE and the diagonal per row, not the
 *                     value array (FP64 and pair-float steps keep the CSR form).  Quantum sun
 *                     (not its default: no faster): FP32 steps take each value from the
 *                     diagonal, the dot block or the ray couplings by the two states' bits.
 *                     The FMA sequence is the CSR step's, so both mappings give the same bits.
 * Errors: PF_EINVAL (unknown mapping, or structured for another model).              */
typedef enum { PF_MAP_CSR = 0, PF_MAP_STRUCTURED = 1 } pf_mapping;
pf_status pf_ham_set_mapping(pf_ham* H, int32_t mapping);

/* Rescaling and the device arrays of H~ values (FP64 and FP32, CSR order).         */
pf_status pf_ham_rescaled(const pf_ham* H, double* Ec, double* dE, const double** val64,
                          const float** val32);

/* Exact moments of the spectrum of H~ from traces: mu~ = Tr H~ / D,
 * G~^2 = Tr H~^2 / D - mu~^2 (Eq. dos_gaussian uses them).  Synchronises.          */
pf_status pf_ham_moments(pf_ham* H, double* mu_t, double* G_t, pf_stream_t stream);

/* (a4) Filter coefficients a_n = c_n/chi, n = 0..K (Eq. transformation,
 * Eq. transformationCoefficients), computed on the device.  coeffs: host [K+1].     */
pf_status pf_filter_coefficients(double lam_t, int32_t K, double* coeffs, pf_stream_t stream);

/* Degree K from the Gaussian DOS with exact moments (Eq. dos_gaussian, Eq. Nev,
 * Eq. K_approx): K = ceil(2.655 sqrt(1 - lam~^2) * 2 rho(lam~) / nev_g),
 * nev_g = ceil(g nev), g = 3 for D >= 100000, else 1.5.
 * target_eps: lambda = Emin + eps (Emax - Emin).  Synchronises. */
pf_status pf_choose_K(pf_ham* H, double target_eps, int32_t nev, int32_t* K, pf_stream_t stream);

/* ---------------------------------------------------------------------------
 * (a5) One fused Clenshaw step (Eq. clenshaw_chebyshev_prod):
 *     out = a * V + alpha * (H~ B1) - beta * B2
 * with alpha = 2 for b_i (i >= 1) and alpha = 1 for the closing line P V = a_0 V +
 * H~ b_1 - b_2.  beta in {0, 1}; B2 may be NULL when beta = 0; out may alias B2
 * (b_i overwrites b_{i+2}); out must not alias V or B1.  alpha = 0 skips the SpMM
 * (B1 may then be NULL).  If use_H is nonzero the unscaled H is used instead of H~
 * (then only precision PF_F64 is allowed).
 *   prec: PF_F64 (double blocks, FP64 values), PF_F32 (float blocks, FP32 values) or
 *         PF_DF64 (pair-float blocks and values; a, alpha, beta are split into pairs).
 *   s   : block width, one of 1, 2, 4, 8, 16, 32, 64.
 * Errors: PF_EINVAL, PF_ESTATE (H~ not set), PF_ECUDA.                             */
pf_status pf_clenshaw_step(const pf_ham* H, int32_t prec, int32_t s, const void* V,
                           const void* B1, const void* B2, void* out, double a, double alpha,
                           double beta, int32_t use_H, pf_stream_t stream);

/* W = P(H~) V for a D x s block: the whole recurrence, K steps, with two internal
 * D x s auxiliary blocks.  coeffs: host [K+1] (FP64 for every precision).  V and W
 * are double blocks for PF_F64, float blocks for PF_F32 and pair-float blocks
 * (D x s x 2 floats) for PF_DF64.                                                  */
pf_status pf_filter_apply(const pf_ham* H, int32_t prec, int32_t s, const void* V, void* W,
                          const double* coeffs, int32_t K, pf_stream_t stream);

/* W_j = P_j(H~_j) V_j for n independent items of one precision and block width (each
 * item its own Hamiltonian, size, coefficients and degree K_j), advanced together: a sweep
 * of max_j(K_j) + 1 launches, each one Clenshaw step of every item over the concatenation
 * of all items' rows.  Item j joins at launch max(K) - K_j, so all items end together.
 * Every row is computed with the operation order of pf_filter_apply, so each W_j is
 * bit-identical to pf_filter_apply on the same item.  The paper applies the filter to one
 * problem at a time; this is the library's batching of many small problems.
 *   items[j].H      : handle with H~ set;  V, W: device blocks (D_j x s) of the precision.
 *   items[j].coeffs : host [K_j + 1];      K: >= 1.
 * Allocates two auxiliary blocks per item, the coefficients and a table of n entries.
 * Errors: PF_EINVAL, PF_ESTATE (H~ not set), PF_ENOMEM, PF_ECUDA (including a cluster
 * shape the device cannot schedule).                                                */
typedef struct {
  const pf_ham* H;
  const void* V;
  void* W;
  const double* coeffs;
  int32_t K;
} pf_filter_item;
/* Execution form of a batch (form argument):
 *   PF_FORM_AUTO  (-1) each item shape's form chosen by the autotuner (pf_filter_tune);
 *   PF_FORM_STEPS  (0) one launch per Clenshaw step over all items' rows;
 *   PF_FORM_GRAPH (-2) the same launches as one CUDA graph (a chain of kernel nodes);
 *   c in {1, 2, 4, 8, 16}: one persistent launch, a thread-block cluster of c CTAs per item
 *      running the item's whole recurrence with a hardware cluster barrier between steps.
 * Every form gives the same bits.                                                    */
#define PF_FORM_AUTO (-1)
#define PF_FORM_STEPS 0
#define PF_FORM_GRAPH (-2)
pf_status pf_filter_apply_batch(const pf_filter_item* items, int32_t n, int32_t prec, int32_t s,
                                int32_t form, pf_stream_t stream);
/* The autotuner's choice for a group of n items shaped like H at (prec, s), degree K:
 * form = 0 (per-step sweep; the plain one-launch-per-step recurrence when n = 1) or a cluster
 * size c >= 1 (persistent).  The shape is measured once per (device, D, nnz, prec, s) on
 * scratch blocks, over min(K, 48) + 1 steps: the item alone with one launch per step, the
 * sweep over enough copies to fill the GPU, and the persistent kernel with clusters of 1, 2,
 * 4, 8, 16 CTAs.  The form with the smallest predicted per-step time for the whole group is
 * chosen: sweep time interpolated between one item and the copies; persistent time x
 * ceil(n / clusters resident at once).  Items with more than 64 rows per thread of a
 * 16-CTA cluster are not measured and take the sweep.
 *   step_us (may be NULL): host [8] = raw, sweep, sweep copies, persistent c = 1, 2, 4, 8, 16
 *   (microseconds per step; 0 = not measured).
 * Errors: PF_EINVAL, PF_ESTATE (H~ not set), PF_ENOMEM, PF_ECUDA.                    */
pf_status pf_filter_tune(const pf_ham* H, int32_t prec, int32_t s, int32_t K, int32_t n, int32_t* form,
                         double* step_us, pf_stream_t stream);

/* W = P_j(H~) v_j column by column: column j of the D x s block takes its own Chebyshev
 * coefficients coeffs[i * s + j], i = 0..K (host, (K+1) x s row-major), in the recurrence of
 * pf_filter_apply (Eq. clenshaw_chebyshev_prod).  The refinement's residual-correction form
 * (PF_REFINE_CORRECTION) runs this recurrence in FP32 on the FP64 residuals.  prec: PF_F64 or
 * PF_F32 (the table is rounded to the filter precision).  Allocates two auxiliary blocks and
 * the device copy of the table.  Errors: PF_EINVAL, PF_ESTATE (H~ not set), PF_ENOMEM,
 * PF_ECUDA.                                                                          */
pf_status pf_filter_apply_cols(const pf_ham* H, int32_t prec, int32_t s, const void* V, void* W,
                               const double* coeffs, int32_t K, pf_stream_t stream);

/* Same computation as pf_filter_apply, without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device memory at
 * the time of the call (a frozen or exhausted memory pool, a host allocator that must not
 * be re-entered from its own hooks, loops that forbid allocation calls).  The two D x s
 * auxiliary blocks come from one fixed device array of 32 MiB inside the library, which
 * every GPU that loads the library keeps until the process exits.
 *  - Limit: 2 * D * s * w <= 32 MiB, w = 8 (PF_F64, PF_DF64) or 4 (PF_F32), each block rounded up
 *    to 256 bytes; larger requests return PF_EINVAL without touching the GPU.
 *  - Every call looks up the array's device address on the current device (a CUDA
 *    symbol query, no allocation), so a context destroyed and re-created in the same
 *    process (cudaDeviceReset) is picked up by the next call.  The first call on a device
 *    may load the library's device code; make it before any stream capture.
 *  - All calls share the array and it keeps the last call's contents (nothing in it needs
 *    to start at zero).  Calls that can overlap on the GPU (other streams, other threads)
 *    race on it; serialise them.
 * Arguments, layout, ownership and the other errors are those of pf_filter_apply.      */
pf_status pf_filter_apply_noalloc(const pf_ham* H, int32_t prec, int32_t s, const void* V, void* W,
                                  const double* coeffs, int32_t K, pf_stream_t stream);

/* ---------------------------------------------------------------------------
 * (a6-a10) The solve: block Lanczos on P(H~) with full reorthogonalisation (two
 * classical Gram-Schmidt passes), shifted Cholesky QR, the block-tridiagonal
 * Lanczos matrix, periodic convergence checks (Eq. blocklan_criterion), Ritz
 * extraction with a Rayleigh-Ritz in H on the converged block, residuals
 * ||H u - E u|| (Sec. 4.3), and, for PF_F32, FP64 refinement passes.
 */
typedef struct {
  int32_t block;          /* s: 1..64, power of two; 0 = 32; < 0 = pf_autotune_block  */
  int32_t precision;      /* pf_precision of the filter recurrence                   */
  int32_t nev_guard;      /* Ritz pairs converged; 0 = ceil(g nev),
                             g = 3 for D >= 100000, else 1.5                        */
  int32_t check_first;    /* first check at this block step; 0 = ceil(m / 2), m the
                             expected Krylov blocks (20.427 s + 1.696 nev_g) / s      */
  int32_t check_every;    /* check interval in block steps; 0 = ceil(m / 10), checked
                             sooner when the largest residual of the last two checks,
                             extrapolated geometrically, reaches tol sooner            */
  int32_t max_blocks;     /* Krylov budget in blocks; 0 = from eta                    */
  double eta;             /* over-allocation of the expected Krylov size; 0 = 1.5    */
  double tol;             /* P-space tolerance on ||B tau|| (FP64 filter); 0 = 1e-10 */
  double tol_f32;         /* same for the FP32 filter stage; 0 = 1e-7                */
  double res_tol;         /* final acceptance ||Hu - Eu|| <= res_tol ||H||; 0 = 1e-9 */
  int32_t refine_passes;  /* FP32 path: max FP64 filter passes; <0 = none, 0 = 8     */
  int32_t refine_K;       /* degree of the refinement filter; 0 = 0.7 K for K >= 1000
                             (back to K after a stalled pass), else K                  */
  uint64_t seed;          /* start block: v[r,c] = SplitMix64(seed, r*s+c) - 1/2     */
  int32_t use_abs_target; /* nonzero: target is target_abs (absolute energy)         */
  double target_abs;
  double refine_shift;    /* shift c of P + cI in refinement passes after the first;
                             0 = 0.05, < 0 = never shift                              */
  int32_t refine_reserve; /* FP32 path: reserve Ritz blocks beyond the guard kept for
                             the refinement set; 0 = 2, < 0 = none                    */
  int32_t refine_full_set;/* nonzero: the reserve blocks are in the refinement set from
                             the first pass (default: one joins per stalled pass)     */
  double refine_guard_lock;/* refinement locks a pair outside the returned set (guard,
                             reserve) once its residual is <= this x res_tol ||H||;
                             0 = 10, < 0 = never (returned pairs: refine_lock)         */
  double refine_lock;     /* refinement locks a returned pair once its residual is <=
                             this x res_tol ||H|| (at most 1); 0 = 0.9                 */
  int32_t refine_precision;/* arithmetic of the refinement filter in the direct form:
                             PF_F64 (the default) or PF_DF64 (pair-float on the FP32
                             units, about 2x faster steps); Gram-Schmidt, Rayleigh-Ritz
                             and the residual check stay FP64 either way               */
  int32_t refine_form;    /* pf_refine_form of the refinement passes; 0 = the default,
                             PF_REFINE_CORRECTION                                      */
  int32_t orth_precision; /* arithmetic of the dense tall-skinny products: the Lanczos
                             stage's two Gram-Schmidt passes, its Cholesky QR products,
                             the Ritz-vector assembly, and the Gram and rotation products
                             of the Rayleigh-Ritz in H and of the refinement's
                             orthonormalisation (SpMMs, residuals, the s x s and q x q
                             factorisations and eigensolves stay FP64):
                             PF_F64, or PF_DF64 (pair-
                             float on the FP32 units, operands and results FP64, about
                             2^-47 relative to the terms' magnitudes; B300 runs FP64 at
                             1/64 of the FP32 rate); 0 = PF_DF64 with the PF_F32 filter,
                             PF_F64 with the PF_F64 filter                             */
} pf_solve_opts;

/* How a refinement pass applies W = (P(H~) + c I) U to a Ritz block U (FP32 filter path).
 *  PF_REFINE_DIRECT      the K-step recurrence on U itself, in refine_precision arithmetic.
 *  PF_REFINE_CORRECTION  residual-correction form: with theta_j = u_j^T H~ u_j and
 *                        beta_i(theta) the recurrence's values on the scalar theta,
 *                        (P(H~) + c) u = (P(theta) + c) u + beta_1 r + H~ d_1 - d_2, where
 *                        r = H~ u - theta u and d_i = 2 beta_{i+1}(theta) r + 2 H~ d_{i+1}
 *                        - d_{i+2}.  r, theta, P(theta) and the final sum are FP64; the d
 *                        recurrence, whose terms are the size of u's error, runs in FP32
 *                        (per-column coefficients), so its rounding adds ~1e-12 relative
 *                        error instead of FP32's ~1e-5: one FP64 SpMM and K FP32 steps per
 *                        pass in place of K FP64 steps.                                  */
typedef enum { PF_REFINE_DIRECT = 1, PF_REFINE_CORRECTION = 2 } pf_refine_form;

typedef struct {
  int32_t status, K, blocks, krylov_dim, nev_guard, converged, checks, refine_passes;
  int64_t filter_steps_f32;    /* FP32 Clenshaw steps (one launch each)                */
  int64_t filter_steps_f64;    /* FP64 Clenshaw steps, Lanczos stage and refinement    */
  double emin, emax, Ec, dE, lambda, lambda_t, hnorm;
  double max_residual;         /* max ||Hu - Eu|| over the returned pairs              */
  double ms_filter_f32;        /* device time of the FP32 filter applications          */
  double ms_filter_f64;        /* device time of the FP64 filter applications          */
  double ms_orth;              /* A_k and the two Gram-Schmidt passes                  */
  double ms_qr;                /* Cholesky QR                                          */
  double ms_check;             /* eigensolves of H_L at the convergence checks         */
  double ms_extract;           /* Ritz vectors, Rayleigh-Ritz in H, residuals          */
  double ms_refine;            /* refinement passes (includes their FP64 filter time)  */
  double ms_total;
  double max_residual_unrefined; /* max ||Hu - Eu|| before any refinement pass         */
  int32_t refine_active[8];    /* blocks filtered in refinement pass p (p < 8)         */
  double refine_residual[8];   /* max ||Hu - Eu|| of the returned pairs after pass p   */
} pf_report;

/* Fill o with the defaults listed in pf_solve_opts.                                */
void pf_default_opts(pf_solve_opts* o);

/*   H          : handle with bounds set (pf_spectral_bounds or pf_set_rescale).
 *   target_eps : normalised energy, lambda = Emin + eps (Emax - Emin), eps in [0,1]
 *                (ignored when o->use_abs_target).
 *   nev        : eigenpairs returned, 1 <= nev <= D.  K: filter degree >= 1.
 *   evals      : host [nev], ascending.      resid: host [nev], ||H u - E u||.
 *   evecs      : device, D x nev column-major (may be NULL).
 *   rep        : host, may be NULL.
 * Synchronises.  Errors: PF_EINVAL, PF_ESTATE, PF_ENOMEM, PF_ENOTCONV (outputs written),
 * PF_EBREAKDOWN, PF_ECUDA.                                                        */
pf_status pf_polfed_solve(pf_ham* H, double target_eps, int32_t nev, int32_t K,
                          const pf_solve_opts* o, double* evals, double* evecs, double* resid,
                          pf_report* rep, pf_stream_t stream);

/* The nev eigenpairs nearest the target of a complex-Hermitian H (Sec. 2: block Lanczos for
 * complex-Hermitian matrices; the model's phi != 0, see pf_model).  The handle holds the real
 * embedding M = [[A, -B], [B, A]] of H = A + iB, whose spectrum is H's with every eigenvalue
 * twice; the call solves M for 2 nev pairs with pf_polfed_solve's path, matches the copies
 * (consecutive values within res_tol ||H||) and returns one eigenpair of H per match: the copy
 * with the smaller residual, its vector [x; y] as z = x + i y (||z|| = 1, ||H z - E z|| equals
 * the copy's residual).  K is the degree for the embedded problem: pf_choose_K(H, eps, 2 nev)
 * puts 2 nev values of M in the window, i.e. nev of H.
 *   evals, resid : host [nev] (ascending).
 *   evecs        : device, D x nev complex, column-major, each entry (re, im) FP64
 *                  (2 D nev doubles; D the sector's dimension); may be NULL.
 * Errors: those of pf_polfed_solve; PF_EINVAL for a real model; PF_EBREAKDOWN when the copies
 * cannot be matched (H has a degenerate eigenvalue among the nev, which this path does not
 * separate).                                                                          */
pf_status pf_polfed_solve_complex(pf_ham* H, double target_eps, int32_t nev, int32_t K,
                                  const pf_solve_opts* o, double* evals, double* evecs, double* resid,
                                  pf_report* rep, pf_stream_t stream);

/* ---------------------------------------------------------------------------
 * (a11) Batched solves: n independent problems (disorder realisations, sizes, targets)
 * solved together.  Every problem is a resumable solve holding its Lanczos state in device
 * memory.  Each round runs the pending filter applications of all unfinished problems
 * (those with the same precision and block width share one sweep, as in
 * pf_filter_apply_batch; the refinement of one problem contributes one item per active
 * block), then each problem's orthogonalisation, QR, checks, extraction or refinement.
 * Each problem's outputs are bit-identical to pf_polfed_solve on the same inputs.  Not in
 * the paper, which solves one problem at a time.                                     */
typedef struct {
  pf_ham* H;                  /* in: handle with bounds set                               */
  double target_eps;          /* in: as pf_polfed_solve                                   */
  int32_t nev, K;             /* in: as pf_polfed_solve                                   */
  const pf_solve_opts* opts;  /* in: NULL = defaults                                      */
  double* evals;              /* out: host [nev], ascending                               */
  double* evecs;              /* out: device D x nev column-major, may be NULL            */
  double* resid;              /* out: host [nev]                                          */
  pf_report* rep;             /* out: host, may be NULL                                   */
  int32_t status;             /* out: this problem's pf_status                            */
} pf_solve_item;
/* Returns PF_OK when every item succeeded, else the first failing item's status; a failed
 * shared launch (PF_ECUDA, PF_ENOMEM) is reported in every item that was running.
 * `stream` is synchronised first; the solves then run on the library's pool of streams
 * (process-wide, 16 streams) and are complete when the call returns.                */
pf_status pf_polfed_solve_batch(pf_solve_item* items, int32_t n, pf_stream_t stream);

/* Device bytes one solve holds at its peak: the Hamiltonian (CSR, FP64 and FP32 H~ copies,
 * basis table) for the given nnz, the resident Lanczos state (basis of the expected Krylov
 * size with eta = 1.5, H_L, work blocks), the Ritz set and, for PF_F32, the refinement
 * blocks.  Used by the server's admission.  Errors: PF_EINVAL.                         */
pf_status pf_solve_footprint(int64_t D, int64_t nnz, int32_t nev, int32_t block, int32_t precision,
                             int64_t* bytes);

/* ---------------------------------------------------------------------------
 * (a12) Serving: continuous batching of solve requests (not in the paper).  Requests are
 * queued on submit.  Each pf_server_step (1) admits queued requests in arrival order while
 * the sum of the admitted footprints (pf_solve_footprint with the model's nnz bound) stays
 * within the budget and fewer than max_active are resident; a request larger than the
 * budget is admitted alone into an empty server; admission builds the basis, Hamiltonian,
 * spectral bounds and K (pf_choose_K) on the server's stream; (2) runs one round of all
 * resident solves as in pf_polfed_solve_batch; (3) retires finished solves, releasing
 * their device memory.  A request's results equal those of the one-problem calls on the
 * same model and options, whatever else is resident.  Not thread-safe: one host thread
 * drives a server.  Latencies are measured on the host's steady clock.               */
typedef struct pf_server pf_server;
typedef struct {
  int32_t block;            /* s of every solve; 0 = 32; < 0 = autotuned per request        */
  int32_t precision;        /* pf_precision of the filter                                  */
  int32_t max_active;       /* most resident solves; 0 = 64                                */
  int64_t mem_budget_bytes; /* admission budget; 0 = 80% of free device memory at create  */
  double res_tol;           /* acceptance ||Hu - Eu|| <= res_tol ||H||; 0 = 1e-9           */
  double bounds_tol;        /* spectral-bounds tolerance; 0 = 1e-10                         */
  uint64_t seed;            /* start-block seed; 0 = 2024                                   */
  int32_t refine_precision; /* refinement filter arithmetic: PF_F64 (0) or PF_DF64          */
  int32_t refine_form;      /* pf_refine_form of the refinement passes; 0 = the default     */
} pf_server_config;
typedef struct {
  int64_t id;
  int32_t status;           /* the request's pf_status                                     */
  int32_t nev;
  int64_t footprint_bytes;  /* admission footprint                                         */
  double queue_ms;          /* submit to admission                                         */
  double latency_ms;        /* submit to completion                                        */
} pf_request_info;
/* cfg may be NULL (defaults).  The resident solves run on the library's pool of streams
 * (one per solve, shared round-robin beyond 16), not on `stream`, which is reserved.
 * Errors: PF_EINVAL, PF_ECUDA.                                                      */
pf_status pf_server_create(const pf_server_config* cfg, pf_stream_t stream, pf_server** out);
/* Queue one request; m and p are copied (host).  id: host output.
 * Errors: PF_EINVAL (model, arrays, eps outside [0,1], nev outside [1, D]; a complex-
 * Hermitian model, phi != 0, which goes through pf_polfed_solve_complex).           */
pf_status pf_server_submit(pf_server* sv, const pf_model* m, const pf_params* p, double target_eps,
                           int32_t nev, int64_t* id);
/* One step as above.  queued / active / finished: host outputs (may be NULL): requests
 * waiting, resident, finished and not yet taken.  Synchronises.  A request that fails
 * (build, bounds, solve) finishes with its status; the call itself returns PF_ECUDA only
 * for a failure of a launch shared by all resident solves.                           */
pf_status pf_server_step(pf_server* sv, int32_t* queued, int32_t* active, int32_t* finished);
/* Results of a finished request, then its record is released.  evals, resid: host [nev]
 * (may be NULL); rep, info: host (may be NULL).  Errors: PF_ESTATE (still queued or
 * resident), PF_EINVAL (unknown or already taken id).                               */
pf_status pf_server_take(pf_server* sv, int64_t id, double* evals, double* resid, pf_report* rep,
                         pf_request_info* info);
/* Sum of the footprints of the resident requests, and the budget.                   */
pf_status pf_server_memory(const pf_server* sv, int64_t* in_use, int64_t* budget);
void pf_server_destroy(pf_server* sv);

/* ---------------------------------------------------------------------------
 * Kernel polynomial method for the density of states (Sec. 3.3, Eq. dos_kpm, App. B).
 * mu_n = Tr T_n(H~), n = 0..N-1, estimated as (1/R) sum_r <r| T_n(H~) |r> over the columns of a
 * D x R random block with entries sqrt(12) (u - 1/2), u the start block's SplitMix64 uniforms
 * (entry (i, r) from counter i R + r; zero mean, unit variance).  Two moments per FP64
 * Clenshaw step (doubling: T_2n = 2 T_n^2 - 1, T_2n+1 = 2 T_n+1 T_n - T_1).
 *   H: handle with H~ set.  R: 1, 2, 4, ..., 64.  mu: host [N].  Synchronises.
 * Errors: PF_EINVAL, PF_ESTATE (H~ not set), PF_ENOMEM, PF_ECUDA.                    */
pf_status pf_kpm_moments(pf_ham* H, int32_t N, int32_t R, uint64_t seed, double* mu, pf_stream_t stream);
/* rho_KPM(x) = [mu_0 g_0 + 2 sum_{n=1}^{N-1} mu_n g_n T_n(x)] / (pi sqrt(1 - x^2)) with the
 * Jackson kernel g_n, at nx points x in (-1, 1) (host arrays).  Errors: PF_EINVAL.     */
pf_status pf_kpm_dos(const double* mu, int32_t N, const double* x, int32_t nx, double* rho);
/* Targets that need the density (Sec. 5.2): E~_maxdos = argmax of rho_KPM on a grid of 4001
 * points in [-0.999, 0.999]; lam_t = E~_maxdos + eta (1 - E~_maxdos) for eta >= 0,
 * E~_maxdos + eta (E~_maxdos + 1) for eta < 0 (eta = 0 is :maxdos, (:offset, eta) otherwise).
 * Errors: PF_EINVAL (eta outside [-1, 1]).                                          */
pf_status pf_kpm_target(const double* mu, int32_t N, double eta, double* lam_t);
/* K from Eq. condition_for_K with rho(lam~) from KPM: delta = nev_g / (2 rho) (Eq. Nev,
 * nev_g = ceil(g nev), g = 3 when mu_0 >= 100000, else 1.5), then the smallest K in
 * [K_approx/2, 2 K_approx] whose filter is at most Omega = sin(2.655)/2.655 at both window
 * edges lam~ +- delta (bisection).
 * Errors: PF_EINVAL (rho <= 0, lam_t outside (-1, 1)).                               */
pf_status pf_choose_K_kpm(const double* mu, int32_t N, double lam_t, int32_t nev, int32_t* K);

/* Block width from the autotuner: the step kernel is timed (8 steps on scratch blocks) for
 * s = 8, 16, 32, 64 and the width with the smallest predicted filter time is returned:
 * ceil(expectedkrylovdim(nev_g, s, 1) / s) x t_step(s) (Sec. 5.5's Krylov-size fit, nev_g =
 * ceil(g nev), g as for pf_choose_K), plus for PF_F32 the FP64 refinement,
 * 1.3 x 0.7 x ceil(nev_g / s) x t_step64(s) (per unit degree); widths above nev_g (and above
 * D/2) are skipped.  Timings are cached per
 * (device, D, nnz, precision).  A solve with block < 0 uses this choice.
 *   step_us, cost: host [4] (may be NULL): measured step time and predicted cost per candidate
 *   (0 = skipped).  Errors: PF_EINVAL, PF_ESTATE (H~ not set), PF_ENOMEM, PF_ECUDA.   */
pf_status pf_autotune_block(pf_ham* H, int32_t precision, int32_t nev, int32_t* block, double* step_us,
                            double* cost, pf_stream_t stream);

/* Start block as the solve draws it: v[r,c] = uniform(SplitMix64(seed, r*s+c)) - 1/2,
 * uniform = top 53 bits * 2^-53 (Steele, Lea & Flood 2014).  out: device double [D*s]. */
pf_status pf_start_block(int64_t D, int32_t s, uint64_t seed, double* out, pf_stream_t stream);

/* Selected eigenpairs of a dense real-symmetric matrix: the eigensolver the solve applies to the
 * projected Lanczos matrix H_L at its convergence checks and its Ritz extraction (Sec. 4.6,
 * Eq. blocklan_criterion).  Householder tridiagonalisation (one thread-block cluster with the matrix
 * in distributed shared memory up to n ~ 620, two launches per column over the GPU up to 3000, four
 * above; every form gives the same tridiagonal bit for bit), multisection with Sturm counts, inverse iteration (Gram-Schmidt within
 * clusters closer than 1e-6 ||T||) and back-transformation, all FP64.
 *   A: device, n x n row-major with leading dimension lda >= n; only (A + A^T) / 2 is used.
 *   idx: host [q], indices into the ascending spectrum (0 = smallest), each in [0, n).
 *   w: host [q], the eigenvalues of those indices.  Z: device, n x q, column k (leading dimension
 *   ldz >= n) the unit eigenvector of w[k].  Allocates its workspace; synchronises the stream.
 * Errors: PF_EINVAL (n < 1, q < 1, q > n, an index outside [0, n), lda or ldz < n, n > 25000),
 * PF_ENOMEM, PF_ECUDA.                                                                     */
pf_status pf_sym_eig_select(const double* A, int32_t lda, int32_t n, const int32_t* idx, int32_t q, double* w,
                            double* Z, int32_t ldz, pf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* POLFED_H */
