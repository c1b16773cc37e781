// Internal definitions shared by the CUDA translation units of libpolfed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <stdio.h>
#include <vector>
#include <atomic>
#include "../../include/polfed.h"

#define PF_MAX_S 64

namespace pf {
// Guard nev_g = ceil(guard_factor(D) nev): the Ritz pairs converged, and the eigenvalues the degree
// K puts above the filter's cutoff (Eq. Nev, Eq. K_approx).  Sectors of D >= 100,000, where the
// filter's matrix products dominate a solve, take 3 (K falls as 1 / nev_g, the Krylov space
// grows only as 20.4 s + 1.7 nev_g); smaller ones, where the Lanczos and Ritz work dominates,
// keep 1.5.  The KPM rule takes D as mu_0 (its estimate of Tr T_0).  The oracle's dos.guard_count
// is the same rule.
inline double guard_factor(double D) { return D >= 100000.0 ? 3.0 : 1.5; }
}  // namespace pf

namespace pf {

// ---------------------------------------------------------------- errors
void set_cuda_error(cudaError_t e, const char* where);

// Number of kernels this library has launched (every launch site counts itself).
extern std::atomic<long long> g_kernel_launches;
#define PF_COUNT(n) (::pf::g_kernel_launches.fetch_add((n), std::memory_order_relaxed))

#define PF_CUDA(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) {                            \
      ::pf::set_cuda_error(_e, #call);                  \
      return PF_ECUDA;                                  \
    }                                                   \
  } while (0)

#define PF_LAUNCH_CHECK(name)                           \
  do {                                                  \
    PF_COUNT(1);                                        \
    cudaError_t _e = cudaGetLastError();                \
    if (_e != cudaSuccess) {                            \
      ::pf::set_cuda_error(_e, name);                   \
      return PF_ECUDA;                                  \
    }                                                   \
  } while (0)

#define PF_TRY(expr)                                    \
  do {                                                  \
    pf_status _s = (expr);                              \
    if (_s != PF_OK) return _s;                         \
  } while (0)

// ---------------------------------------------------------------- memory
void* dev_alloc(size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);

// RAII owner of one device allocation (internal scratch).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  pf_status alloc(size_t nbytes, cudaStream_t stream) {
    release();
    st = stream;
    bytes = nbytes;
    if (nbytes == 0) return PF_OK;
    p = dev_alloc(nbytes, stream);
    return p ? PF_OK : PF_ENOMEM;
  }
  void release() {
    if (p) dev_free(p, st);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline bool valid_prec(int prec) { return prec == PF_F64 || prec == PF_F32 || prec == PF_DF64; }
// bytes per block entry of a filter precision (a pair-float entry is two floats)
inline size_t prec_bytes(int prec) { return prec == PF_F32 ? 4 : 8; }

// ---------------------------------------------------------------- handles
struct Basis {
  pf_model m;
  int64_t D = 0, D_up = 0, D_dn = 0;
  uint32_t* states = nullptr;   // device
  uint64_t* binom = nullptr;    // device, 33 x 33, binom[n*33+k]
  cudaStream_t st = 0;
};

struct Ham {
  pf_model m;
  int64_t D = 0, nnz = 0;
  int64_t Dc = 0;               // complex-Hermitian model: its dimension (D = 2 Dc, the real embedding)
  int64_t* row_ptr = nullptr;   // device [D+1]
  int32_t* col = nullptr;       // device [nnz]
  double* val = nullptr;        // device [nnz], H
  double* val_t = nullptr;      // device [nnz], H~ (FP64)
  float* val32 = nullptr;       // device [nnz], H~ (FP32)
  float2* val_df = nullptr;     // device [nnz], H~ as pair-float (hi, lo), hi = val32
  // structured mapping (QREM): the diagonal of H~ per row in the three forms, and the one
  // off-diagonal value (-Gamma / dE); the steps then read no CSR arrays
  int mapping = PF_MAP_CSR;
  double* diag_t = nullptr;
  float* diag32 = nullptr;
  float2* diag_df = nullptr;
  double off_t = 0.0;
  // quantum sun: the dot block (2^N x 2^N) and the ray couplings (L) of H, kept on the host at
  // build, and of H~ on the device after the rescale (one array per precision: qtab_n block
  // entries, then the couplings)
  std::vector<double> qs_hdot, qs_coef;
  double* qtab_t = nullptr;
  float* qtab32 = nullptr;
  float2* qtab_df = nullptr;
  int qtab_n = 0;
  int has_rescale = 0, has_bounds = 0;
  double Ec = 0, dE = 1, emin = 0, emax = 0, rmin = 0, rmax = 0, hnorm = 0;
  cudaStream_t st = 0;
};

// binomial table n, k <= 32 (host)
void host_binom(uint64_t* tab /*33*33*/);

// ---------------------------------------------------------------- device helpers
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic block-wide sum (power-of-two blockDim <= 1024); result valid in all threads.
template <typename T>
__device__ T block_sum(T v, T* sh /* >= 32 */) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (w == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- cross-unit API
// The matrix values a step of precision prec reads: H~ in FP64, FP32 or pair-float.
inline const void* ham_vals(const Ham* H, int prec) {
  return prec == PF_F64 ? (const void*)H->val_t : prec == PF_F32 ? (const void*)H->val32 : (const void*)H->val_df;
}

// Clenshaw step on raw CSR arrays (clenshaw.cu)
// cta_cap > 0 limits the step's CTAs per SM (room for another solve's kernels beside it).
// acol (device, s values in the step's precision, FP64 or FP32), when not null, gives each
// column of the block its own coefficient in place of a.
pf_status clenshaw_step_raw(int64_t D, const int64_t* row_ptr, const int32_t* col, const void* val,
                            int prec, int s, const void* V, const void* B1, const void* B2, void* out,
                            double a, double alpha, double beta, cudaStream_t st, int cta_cap = 0,
                            const void* acol = nullptr);
// One step of H~ through the handle's mapping (CSR arrays or the structured QREM rows); the
// operands and errors of clenshaw_step_raw.
pf_status ham_step(const Ham* H, int prec, int s, const void* V, const void* B1, const void* B2, void* out,
                   double a, double alpha, double beta, cudaStream_t st, int cta_cap = 0, const void* acol = nullptr);
// One filter application W = P(H~) V (K steps) with its own two auxiliary blocks.
struct FilterItem {
  const Ham* H = nullptr;
  int prec = 0, s = 0;
  const void* V = nullptr;
  void* W = nullptr;
  const double* coeffs_host = nullptr;  // host, K+1 (single-item path)
  const double* coeffs_dev = nullptr;   // device, K+1 (sweeps)
  int K = 0;
  void* aux0 = nullptr;
  void* aux1 = nullptr;
  const void* owner = nullptr;          // the solve the item belongs to (grouping only)
  struct FilterGraph* graph = nullptr;  // the owner's captured form of this application (async executor)
  int cta_cap = 0;                      // CTAs per SM for its steps (0 = all that fit)
  // device, (K+1) x s: a coefficient per column and step in place of coeffs (the refinement's
  // residual-correction form).  Such an item runs alone (plain recurrence or its captured
  // graph), never in a sweep or persistent launch.
  const void* colcoef = nullptr;
};
// A per-step sweep captured as a CUDA graph (chain of T kernel nodes), reused while the table
// address, item count, step count and row total stay the same.
struct SweepGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int prec = -1, s = 0, n = 0, T = 0;
  int64_t rows = 0;
  bool uniform = false;
  const void* table = nullptr;
  SweepGraph() = default;
  SweepGraph(const SweepGraph&) = delete;
  SweepGraph& operator=(const SweepGraph&) = delete;
  ~SweepGraph();
  void reset();
};
// All items (same prec and s) advance together.  csize = 0: one launch per Clenshaw step over
// the concatenated rows (through `graph` when given); csize >= 1: one persistent launch, one
// cluster of csize CTAs per item.  table_host/table_dev: room for filter_sweep_table_bytes(n).
pf_status filter_sweep(const std::vector<FilterItem>& items, void* table_dev, size_t table_bytes, void* table_host,
                       cudaStream_t st, int csize = 0, SweepGraph* graph = nullptr);
size_t filter_sweep_table_bytes(int n);
// Autotuner measurements for one item shape (per-step microseconds; 0 = not measured): the
// item alone with one launch per step, the per-step sweep over sweep_copies copies, and the
// persistent kernel with clusters of 1, 2, 4, 8, 16 CTAs (slots of them run at once).
struct TuneResult {
  double raw_us = 0, sweep_us = 0;
  int sweep_copies = 1;
  double persist_us[5] = {0, 0, 0, 0, 0};
  int slots[5] = {0, 0, 0, 0, 0};
};
// The fastest form for a group of n items of the measured shape: 0 = sweep (the plain
// recurrence when n = 1), c >= 1 = persistent with clusters of c CTAs.
int choose_form(const TuneResult& tr, int n, double* predicted_us);
pf_status tune_item(const FilterItem& it, cudaStream_t st, TuneResult* out);
// A filter application captured as a CUDA graph (see clenshaw.cu); replayed while its
// operands and end coefficients are unchanged, recaptured otherwise.
struct FilterGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int K = -1, prec = -1, s = 0;
  const void* V = nullptr;
  const void* W = nullptr;
  const void* aux0 = nullptr;
  const void* aux1 = nullptr;
  const Ham* H = nullptr;
  double a0 = 0, aK = 0;
  int cap = 0;
  const void* colcoef = nullptr;
  FilterGraph() = default;
  FilterGraph(const FilterGraph&) = delete;
  FilterGraph& operator=(const FilterGraph&) = delete;
  ~FilterGraph();
  void reset();
};
pf_status filter_graph_launch(FilterGraph& g, const FilterItem& it, cudaStream_t st);
// Device coefficient table of a filter precision, n entries of 8 bytes: the values, or for
// PF_DF64 their (hi, lo) float pairs (the form the sweep and persistent kernels read).
void coeff_table_host(int prec, const double* c, int n, double* out);
// W = P V for a D x s block (K steps); aux buffers are two D x s blocks of the filter type.
// colcoef (device, (K+1) x s values of the filter precision, FP64 or FP32), when not null,
// replaces coeffs_host: every column takes its own coefficient of each step.
pf_status filter_apply_raw(const Ham* H, int prec, int s, const void* V, void* W, const double* coeffs_host,
                           const void* colcoef, int K, void* aux0, void* aux1, cudaStream_t st, int cta_cap = 0);

// Dense tall-skinny kernels (dense.cu).  Blocked storage: nb blocks, each D x s row-major,
// block b at X + b*D*s.
// C[nbX*s x nbY*s] (row-major, ldc = nbY*s) = X^T Y  (two-stage deterministic reduction)
pf_status gram(int64_t D, int s, const double* X, int nbX, const double* Y, int nbY, double* C,
               double* scratch, size_t scratch_elems, cudaStream_t st);
size_t gram_scratch_elems(int64_t D, int s, int nbX, int nbY);
// Y(nbY blocks) = beta*Y + alpha * X(nbX blocks) * C, C row-major (nbX*s) x (nbY*s), ldc >= nbY*s.
// Y may equal X only when nbX == nbY == 1.
pf_status tsgemm(int64_t D, int s, const double* X, int nbX, const double* C, int ldc, double* Y, int nbY,
                 double alpha, double beta, cudaStream_t st);
// The same two products in pair-float arithmetic on the FP32 units (operands and results FP64;
// each product and sum carried as an unevaluated float pair, about 2^-47 relative to the sum of
// the terms' magnitudes).  s = 16, 32, 64; other s run the FP64 kernels above.
pf_status gram_df(int64_t D, int s, const double* X, int nbX, const double* Y, int nbY, double* C,
                  double* scratch, size_t scratch_elems, cudaStream_t st);
pf_status tsgemm_df(int64_t D, int s, const double* X, int nbX, const double* C, int ldc, double* Y, int nbY,
                    double alpha, double beta, cudaStream_t st);
// gram_df with Y already split into (hi, lo) float pairs by convert_d2df (s = 16, 32, 64 only):
// the same result, with the Y blocks split once instead of once per X block.
pf_status gram_df_ysplit(int64_t D, int s, const double* X, int nbX, const float2* Y, int nbY, double* C,
                         double* scratch, size_t scratch_elems, cudaStream_t st);
// Column norms of R = A - B*diag(e) for nb blocks (norms[nb*s]); B may be NULL (then ||A||)
pf_status colnorms(int64_t D, int s, const double* A, const double* B, const double* e, int nb, double* norms,
                   double* scratch, size_t scratch_elems, cudaStream_t st);
// Conversions between double and float blocks
pf_status convert_d2f(const double* x, float* y, int64_t n, cudaStream_t st);
pf_status convert_f2d(const float* x, double* y, int64_t n, cudaStream_t st);
// Between double and pair-float blocks (n entries): hi = rn(x), lo = rn(x - hi); back: hi + lo.
// x and y may be the same buffer (both 8 bytes per entry).
pf_status convert_d2df(const double* x, float2* y, int64_t n, cudaStream_t st);
pf_status convert_df2d(const float2* x, double* y, int64_t n, cudaStream_t st);
// Small dense helpers on one CTA
// Shifted Cholesky of G (n x n, row-major), writes upper R (row-major) with G + shift*I = R^T R;
// Rinv = R^{-1} (upper); status[0] = 0 ok, 1 = not positive definite.
pf_status small_chol_inv(const double* G, int n, double shift_rel, double* R, double* Rinv, int* status,
                         cudaStream_t st);
// Rout = A * B (n x n, upper triangular products, row-major)
pf_status small_matmul(const double* A, const double* B, double* C, int n, cudaStream_t st);

// Symmetric eigensolver for a dense n x n matrix (eig.cu).  Computes the eigenvalues with
// indices [lo, hi) of the ascending order and their eigenvectors (columns of Z, ldz = n).
struct EigWork;
size_t eig_workspace_bytes(int nmax, int qmax);
pf_status sym_eig_range(const double* A, int lda, int n, int lo, int hi, double* w_host, double* Z_dev,
                        void* work, size_t work_bytes, cudaStream_t st);

// Seeded start block (solver.cu)
pf_status start_block_raw(int64_t D, int s, uint64_t seed, double* out, cudaStream_t st);

}  // namespace pf
