// (a3) spectral bounds, (a4) coefficients, (a6-a10) the POLFED block-Lanczos solve.
//
// Block Lanczos (paper Sec. 2.2 and Sec. 4.3) on an operator Op:
//     W_k = Op V_k;  A_k = V_k^T W_k;
//     W_k -= V_{1:k} (V_{1:k}^T W_k)     twice (classical Gram-Schmidt, full reorth.);
//     W_k = V_{k+1} B_{k+1}              shifted Cholesky QR (three passes);
//     H_L: A_k on the diagonal, B_{k+1} below, B_{k+1}^T above.
// Convergence (Eq. blocklan_criterion): at checkpoints the selected eigenpairs (theta_j,
// t_j) of H_L must satisfy ||B_{k+1} tau_kj|| <= tol, tau_kj the last block of t_j.
//   Op = H (FP64)            spectral bounds, selected pairs = the two extremes;
//   Op = P(H~) (Clenshaw)    the solve, selected pairs = the nev_g largest theta.
// Extraction (Sec. 4.3): U = V_{1:m} T_sel, then a Rayleigh-Ritz with H on span(U)
// (separates Ritz vectors whose filter values nearly coincide), residuals
// ||H u - E u||, and the nev pairs nearest lambda.  With the FP32 filter the Krylov
// basis and everything after the filter stay FP64, and FP64 filter passes
// (U <- P(H~) U, Cholesky QR, Rayleigh-Ritz) refine the pairs until
// ||H u - E u|| <= res_tol ||H||.
#include "common.cuh"
#include <cmath>
#include <algorithm>
#include <numeric>
#include <chrono>
#include <array>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>

namespace pf {

pf_status set_rescale(Ham* H, double Ec, double dE, cudaStream_t st);
pf_status ham_moments(Ham* H, double* mu_t, double* G_t, cudaStream_t st);
pf_status sym_eig_select(const double* A, int lda, int n, const int* idx_host, int q, double* w_host, double* Z,
                         int ldz, void* work, size_t work_bytes, cudaStream_t st);

// ------------------------------------------------------------------ small kernels
__device__ __forceinline__ double splitmix_unit(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void start_block_kernel(int64_t n, uint64_t seed, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = splitmix_unit(seed, (uint64_t)i) - 0.5;
}

pf_status start_block_raw(int64_t D, int s, uint64_t seed, double* out, cudaStream_t st) {
  const int64_t n = D * s;
  start_block_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(n, seed, out);
  PF_LAUNCH_CHECK("start_block_kernel");
  return PF_OK;
}

// a_n = c_n / chi, c_0 = 1, c_n = 2 cos(n arccos lam~), chi = sum_n c_n cos(n arccos lam~)
__global__ void coeff_kernel(double lam_t, int K, double* c, double* t) {
  const double th = acos(lam_t);
  for (int n = threadIdx.x; n <= K; n += blockDim.x) {
    double T = cos((double)n * th);
    t[n] = T;
    c[n] = (n == 0 ? 1.0 : 2.0) * T;
  }
}
__global__ void coeff_norm_kernel(int K, double* c, const double* t) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int n = threadIdx.x; n <= K; n += blockDim.x) s += c[n] * t[n];
  s = block_sum(s, sh);
  for (int n = threadIdx.x; n <= K; n += blockDim.x) c[n] /= s;
}

static pf_status filter_coefficients_dev(double lam_t, int K, double* host, cudaStream_t st) {
  DevBuf b;
  PF_TRY(b.alloc((size_t)2 * (K + 1) * sizeof(double), st));
  coeff_kernel<<<1, 1024, 0, st>>>(lam_t, K, b.as<double>(), b.as<double>() + K + 1);
  coeff_norm_kernel<<<1, 1024, 0, st>>>(K, b.as<double>(), b.as<double>() + K + 1);
  PF_COUNT(1);
  PF_LAUNCH_CHECK("coeff_kernel");
  PF_CUDA(cudaMemcpyAsync(host, b.p, (K + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  PF_CUDA(cudaStreamSynchronize(st));
  return PF_OK;
}

// HL[(k+1)s.., k s..] = B, HL[k s.., (k+1)s..] = B^T, and optionally the diagonal block A (symmetrised).
__global__ void hl_store_kernel(double* HL, int ld, int k, int s, const double* A, const double* B) {
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) {
    int a = i / s, b = i % s;
    if (A) HL[(int64_t)(k * s + a) * ld + k * s + b] = 0.5 * (A[a * s + b] + A[b * s + a]);
    if (B) {
      HL[(int64_t)((k + 1) * s + a) * ld + k * s + b] = B[a * s + b];
      HL[(int64_t)(k * s + b) * ld + (k + 1) * s + a] = B[a * s + b];
    }
  }
}

// res[j] = || B * Z[n-s:n, j] || for the q columns of Z (column-major, ldz)
__global__ void block_resid_kernel(const double* B, int s, const double* Z, int ldz, int n, int q, double* res) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= q) return;
  const double* tau = Z + (int64_t)j * ldz + (n - s);
  double acc = 0.0;
  for (int a = 0; a < s; ++a) {
    double r = 0.0;
    for (int b = a; b < s; ++b) r = fma(B[a * s + b], tau[b], r);
    acc = fma(r, r, acc);
  }
  res[j] = sqrt(acc);
}

// C (n x q row-major, ldc) = Z (n x q column-major, ldz) with column order perm (C col c = Z col perm[c])
__global__ void z_to_rowmajor_kernel(const double* Z, int ldz, int n, int q, const int* perm, double* C, int ldc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * q) return;
  int r = (int)(i / q), c = (int)(i % q);
  C[(int64_t)r * ldc + c] = Z[(int64_t)perm[c] * ldz + r];
}

// out column c = in column perm[c], both blocked D x s storage, q columns
__global__ void permute_cols_kernel(int64_t D, int s, const double* in, const int* perm, int q, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= D * q) return;
  int c = (int)(i % q);
  int64_t r = i / q;
  int p = perm[c];
  out[(int64_t)(c / s) * D * s + r * s + (c % s)] = in[(int64_t)(p / s) * D * s + r * s + (p % s)];
}

// evecs[:, j] (column-major D x nev) = U column sel[j] (blocked D x s storage)
// ---- residual-correction form of a refinement pass (PF_REFINE_CORRECTION)
// For a column u with theta = u^T H~ u, let beta_i be the recurrence's values on the scalar theta,
// beta_i = a_i + 2 theta beta_{i+1} - beta_{i+2} (beta_{K+1} = beta_{K+2} = 0).  Subtracting
// beta_i u from the vector recurrence leaves d_i = b_i - beta_i u with
//   d_i = 2 beta_{i+1} r + 2 H~ d_{i+1} - d_{i+2},  r = H~ u - theta u,
// and P(H~) u = P(theta) u + beta_1 r + H~ d_1 - d_2, P(theta) = a_0 + theta beta_1 - beta_2.
// The d recurrence is a Clenshaw recurrence of degree K - 1 on r with per-column coefficients
// gamma_0 = beta_1, gamma_i = 2 beta_{i+1} (i >= 1).  One thread per column: theta from the
// diagonal of C = U^T (H~ U), the gamma table (FP32, K rows of s), P(theta) (a[0] already holds
// the pass's shift c) and theta.
__global__ void corr_table_kernel(const double* a, int K, const double* C, int s, float* gamma, double* p,
                                  double* theta) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= s) return;
  const double th = C[(int64_t)j * s + j];
  double b1 = 0.0, b2 = 0.0;   // beta_{i+1}, beta_{i+2}
  for (int i = K; i >= 1; --i) {
    const double bi = fma(2.0 * th, b1, a[i] - b2);
    if (i >= 2) gamma[(int64_t)(i - 1) * s + j] = (float)(2.0 * bi);
    b2 = b1;
    b1 = bi;
  }
  gamma[j] = (float)b1;
  p[j] = a[0] + th * b1 - b2;
  theta[j] = th;
}

// r (FP32) = H~ U - theta U, column j scaled by theta[j]; H~ U and U are FP64 D x s row-major.
__global__ void corr_resid_kernel(int64_t n, int s, const double* HU, const double* U, const double* theta,
                                  float* r) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = (float)(HU[i] - theta[i % s] * U[i]);
}

// W (FP64) = P(theta) U + dW, dW the FP32 result of the d recurrence's closing line.
__global__ void corr_combine_kernel(int64_t n, int s, const double* U, const double* p, const float* dW, double* W) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  W[i] = fma(p[i % s], U[i], (double)dW[i]);
}

__global__ void gather_cols_kernel(int64_t D, int s, const double* U, const int* sel, int nev, double* out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= D * nev) return;
  int j = (int)(i / D);
  int64_t r = i % D;
  int c = sel[j];
  out[i] = U[(int64_t)(c / s) * D * s + r * s + (c % s)];
}

// ------------------------------------------------------------------ workspace
struct Solver {
  const Ham* H = nullptr;
  cudaStream_t st = 0;
  int64_t D = 0;
  int s = 0, max_blocks = 0, Mcap = 0;
  DevBuf V, HL, W, tmp, aux0, aux1, V32, W32, small, gscr, eigw, Z, Cg;
  size_t gscr_elems = 0, eig_bytes = 0;
  int qmax = 0;
  // small: A, B, G, R, Rinv, R2.., status
  double *Ab, *Bb, *Gb, *Rb, *Rib, *R1, *R2, *R3, *T1, *res;
  int* stat;
  pf_report rep;
  cudaEvent_t ev[2];
  bool df = false;   // Cholesky QR's Gram product and update in pair-float (the FP32 path)
};

static pf_status solver_init(Solver& S, const Ham* H, int s, int max_blocks, int qmax, bool f32, cudaStream_t st) {
  S.H = H;
  S.st = st;
  S.D = H->D;
  S.s = s;
  S.max_blocks = max_blocks;
  S.Mcap = (max_blocks + 1) * s;
  S.qmax = qmax;
  const int64_t blk = S.D * s;
  PF_TRY(S.V.alloc((size_t)(max_blocks + 1) * blk * 8, st));
  PF_TRY(S.HL.alloc((size_t)S.Mcap * S.Mcap * 8, st));
  PF_CUDA(cudaMemsetAsync(S.HL.p, 0, (size_t)S.Mcap * S.Mcap * 8, st));
  PF_TRY(S.W.alloc(blk * 8, st));
  PF_TRY(S.tmp.alloc(blk * 8, st));
  if (f32) {
    PF_TRY(S.aux0.alloc(blk * 4, st));
    PF_TRY(S.aux1.alloc(blk * 4, st));
    PF_TRY(S.V32.alloc(blk * 4, st));
    PF_TRY(S.W32.alloc(blk * 4, st));
  } else {
    PF_TRY(S.aux0.alloc(blk * 8, st));
    PF_TRY(S.aux1.alloc(blk * 8, st));
  }
  // Gram scratch: the largest of (max_blocks+1) x 1 blocks and qmax/s x qmax/s blocks
  int qb = (qmax + s - 1) / s;
  size_t g1 = gram_scratch_elems(S.D, s, max_blocks + 1, 1);
  size_t g2 = gram_scratch_elems(S.D, s, qb, qb);
  size_t g3 = (size_t)256 * (qb + 2) * s;   // colnorms
  S.gscr_elems = std::max(std::max(g1, g2), g3);
  PF_TRY(S.gscr.alloc(S.gscr_elems * 8, st));
  const int nsm = 10;
  PF_TRY(S.small.alloc((size_t)nsm * s * s * 8 + (size_t)(qmax + S.Mcap) * 8 + 64, st));
  double* b = S.small.as<double>();
  S.Ab = b; S.Bb = b + s * s; S.Gb = b + 2 * s * s; S.Rb = b + 3 * s * s; S.Rib = b + 4 * s * s;
  S.R1 = b + 5 * s * s; S.R2 = b + 6 * s * s; S.R3 = b + 7 * s * s; S.T1 = b + 8 * s * s;
  S.res = b + nsm * s * s;
  S.stat = (int*)(S.res + qmax + S.Mcap);
  S.eig_bytes = eig_workspace_bytes(S.Mcap, std::max(qmax, 2));
  PF_TRY(S.eigw.alloc(S.eig_bytes, st));
  PF_TRY(S.Z.alloc((size_t)S.Mcap * std::max(qmax, 2) * 8, st));
  // coefficient matrix for CGS (Mcap x s) and for Ritz rotation (Mcap x qmax)
  PF_TRY(S.Cg.alloc((size_t)S.Mcap * std::max(qmax, s) * 8, st));
  memset(&S.rep, 0, sizeof(S.rep));
  return PF_OK;
}

static double* blockp(const Solver& S, int k) { return S.V.as<double>() + (int64_t)k * S.D * S.s; }

// Shifted Cholesky QR, three passes (shift only in the first).  In: X (D x s, FP64, may be
// overwritten), out: Q (D x s), R (s x s upper, into S.Bb).  Returns PF_EBREAKDOWN when the
// factorisation fails.
static pf_status chol_qr3(Solver& S, double* X, double* Q) {
  const int s = S.s;
  const double u = 1.1102230246251565e-16;
  const double shift = 11.0 * ((double)S.D * s + (double)s * (s + 1)) * u;
  double* Rs[3] = {S.R1, S.R2, S.R3};
  double* src = X;
  for (int pass = 0; pass < 3; ++pass) {
    PF_TRY((S.df ? gram_df : gram)(S.D, s, src, 1, src, 1, S.Gb, S.gscr.as<double>(), S.gscr_elems, S.st));
    PF_TRY(small_chol_inv(S.Gb, s, pass == 0 ? shift : 0.0, Rs[pass], S.Rib, S.stat + pass, S.st));
    PF_TRY((S.df ? tsgemm_df : tsgemm)(S.D, s, src, 1, S.Rib, s, S.tmp.as<double>(), 1, 1.0, 0.0, S.st));
    PF_CUDA(cudaMemcpyAsync(Q, S.tmp.p, (size_t)S.D * s * 8, cudaMemcpyDeviceToDevice, S.st));
    src = Q;
  }
  // one read of the three passes' status words (a failed pass substitutes 1 for a non-positive
  // pivot, so the later passes run on finite values; Q and R are then discarded by the caller)
  int bad[3] = {0, 0, 0};
  PF_CUDA(cudaMemcpyAsync(bad, S.stat, sizeof(bad), cudaMemcpyDeviceToHost, S.st));
  PF_CUDA(cudaStreamSynchronize(S.st));
  if (bad[0] || bad[1] || bad[2]) return PF_EBREAKDOWN;
  // R = R3 R2 R1
  PF_TRY(small_matmul(S.R3, S.R2, S.T1, s, S.st));
  PF_TRY(small_matmul(S.T1, S.R1, S.Bb, s, S.st));
  return PF_OK;
}

enum OpKind { OP_H = 0, OP_FILTER64 = 1, OP_FILTER32 = 2 };

static pf_status apply_op(Solver& S, OpKind op, const double* Vk, double* Wk, const double* coeffs, int K) {
  const Ham* H = S.H;
  if (op == OP_H) {
    return clenshaw_step_raw(S.D, H->row_ptr, H->col, H->val, PF_F64, S.s, Vk, Vk, nullptr, Wk, 0.0, 1.0, 0.0, S.st);
  }
  if (op == OP_FILTER64) {
    S.rep.filter_steps_f64 += K + 1;
    return filter_apply_raw(H, PF_F64, S.s, Vk, Wk, coeffs, nullptr, K, S.aux0.p, S.aux1.p, S.st);
  }
  S.rep.filter_steps_f32 += K + 1;
  const int64_t n = S.D * S.s;
  PF_TRY(convert_d2f(Vk, S.V32.as<float>(), n, S.st));
  PF_TRY(filter_apply_raw(H, PF_F32, S.s, S.V32.p, S.W32.p, coeffs, nullptr, K, S.aux0.p, S.aux1.p, S.st));
  return convert_f2d(S.W32.as<float>(), Wk, n, S.st);
}

// Device-time accounting of the solve's phases: events recorded on the solve's stream,
// read back when the phase's last event has completed.
struct PhaseClock {
  cudaEvent_t ev[8];
  cudaStream_t st;
  explicit PhaseClock(cudaStream_t s) : st(s) {
    for (auto& e : ev) cudaEventCreate(&e);
  }
  ~PhaseClock() {
    for (auto& e : ev) cudaEventDestroy(e);
  }
  void mark(int i) { cudaEventRecord(ev[i], st); }
  double ms(int a, int b) {
    float t = 0;
    cudaEventSynchronize(ev[b]);
    cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
};

// Modelled device time (us) of a convergence check and of a block step, from sizes alone.  They
// decide where the next check falls, which decides the Krylov dimension a solve stops at, so they
// must not come from measured times: a solve sharing the GPU with others (a batch, the server) then
// takes the same steps, and returns the same bits, as the same solve alone.  The rates are those the
// kernels reach on B300: the Clenshaw step at ~4 TB/s of its algorithmic bytes (FP64: ~1 TFLOP/s on
// the FP64 pipe), the Gram products at ~1 TFLOP/s, a floor of a few us per dependent launch; the
// eigensolver's tridiagonalisation ~M (3 + 0.0135 M) us, the Sturm counts ~3 M us, inverse iteration
// and back-transformation ~0.03 q M us, ~150 us of launches and host reads per check.
static double model_check_us(int M, int q) {
  return 150.0 + (double)M * (6.0 + 0.0135 * (double)M) + 0.03 * (double)q * (double)M;
}
static double model_block_us(const Ham* H, int s, int K, int k, bool fp64_step) {
  const double D = (double)H->D, nnz = (double)H->nnz, ss = (double)s * (double)s;
  const double w = fp64_step ? 8.0 : 4.0;
  const double bytes = nnz * (w + 4.0) + 8.0 * (D + 1.0) + 4.0 * D * s * w;
  double step = std::max(4.0, bytes / 4.0e6);
  if (fp64_step) step = std::max(step, 2.0 * nnz * s / 1.0e6);
  const double orth = std::max(24.0, 8.0 * (double)(k + 1) * ss * D / 1.0e6);
  const double qr = std::max(60.0, 6.0 * ss * D / 1.0e6);
  return (double)(K + 1) * step + orth + qr;
}

struct LanczosResult {
  int blocks = 0;      // number of Krylov blocks in the basis (M = blocks * s)
  bool converged = false;
  std::vector<double> theta;   // selected Ritz values (ascending)
  std::vector<int> idx;        // their indices in the ascending order of H_L's spectrum
  std::vector<double> resid;
};

// Runs block Lanczos from the start block already in V[0].  select: 0 = extremes, 1 = top q.
static pf_status block_lanczos(Solver& S, OpKind op, const double* coeffs, int K, int select, int q, int min_M,
                               double tol, bool tol_relative, int check_first, int check_every, LanczosResult& out) {
  const int s = S.s;
  const int64_t D = S.D;
  PhaseClock clk(S.st);
  int k = 0;
  int next_check = check_first, prev_k = 0;
  double prev_r = 0.0;
  for (;;) {
    double* Vk = blockp(S, k);
    double* W = S.W.as<double>();
    clk.mark(0);
    PF_TRY(apply_op(S, op, Vk, W, coeffs, K));
    clk.mark(1);
    // A_k = V_k^T W
    PF_TRY(gram(D, s, Vk, 1, W, 1, S.Ab, S.gscr.as<double>(), S.gscr_elems, S.st));
    hl_store_kernel<<<1, 256, 0, S.st>>>(S.HL.as<double>(), S.Mcap, k, s, S.Ab, nullptr);
    PF_LAUNCH_CHECK("hl_store_kernel");
    // full reorthogonalisation, two classical Gram-Schmidt passes
    for (int pass = 0; pass < 2; ++pass) {
      PF_TRY(gram(D, s, S.V.as<double>(), k + 1, W, 1, S.Cg.as<double>(), S.gscr.as<double>(), S.gscr_elems, S.st));
      PF_TRY(tsgemm(D, s, S.V.as<double>(), k + 1, S.Cg.as<double>(), s, W, 1, -1.0, 1.0, S.st));
    }
    clk.mark(2);
    // full: the basis spans the whole space, so B_{k+1} = 0 exactly.  cap: no room for
    // another block; B_{k+1} comes from the Cholesky factor of W^T W alone (enough for
    // ||B tau||), and the iteration stops.
    const bool full = (int64_t)(k + 1) * s >= D;
    const bool cap = (int64_t)(k + 2) * s > D;
    const bool exhausted = full || cap;
    if (full) {
      PF_CUDA(cudaMemsetAsync(S.Bb, 0, (size_t)s * s * 8, S.st));
    } else if (cap) {
      const double u = 1.1102230246251565e-16;
      PF_TRY(gram(D, s, W, 1, W, 1, S.Gb, S.gscr.as<double>(), S.gscr_elems, S.st));
      PF_TRY(small_chol_inv(S.Gb, s, 11.0 * ((double)D * s + (double)s * (s + 1)) * u, S.Bb, S.Rib, S.stat, S.st));
    } else {
      pf_status qs = chol_qr3(S, W, blockp(S, k + 1));
      if (qs != PF_OK) return qs;
    }
    hl_store_kernel<<<1, 256, 0, S.st>>>(S.HL.as<double>(), S.Mcap, k, s, nullptr, S.Bb);
    PF_LAUNCH_CHECK("hl_store_kernel");
    clk.mark(3);
    (op == OP_FILTER32 ? S.rep.ms_filter_f32 : S.rep.ms_filter_f64) += clk.ms(0, 1);
    S.rep.ms_orth += clk.ms(1, 2);
    S.rep.ms_qr += clk.ms(2, 3);
    ++k;
    const int M = k * s;
    const bool last = (k + 1 > S.max_blocks) || exhausted;
    const bool enough = (select == 0 ? M >= 2 : M >= q) && M >= min_M;
    const bool at_check = k >= next_check || last;
    if (enough && at_check) {
      std::vector<int> idx;
      if (select == 0) {
        idx.push_back(0);
        if (M > 1) idx.push_back(M - 1);
      } else {
        for (int i = M - q; i < M; ++i) idx.push_back(i);
      }
      const int nq = (int)idx.size();
      std::vector<double> th(nq), res(nq);
      clk.mark(4);
      PF_TRY(sym_eig_select(S.HL.as<double>(), S.Mcap, M, idx.data(), nq, th.data(), S.Z.as<double>(), M,
                            S.eigw.p, S.eig_bytes, S.st));
      block_resid_kernel<<<(unsigned)ceil_div(nq, 64), 64, 0, S.st>>>(S.Bb, s, S.Z.as<double>(), M, M, nq, S.res);
      PF_LAUNCH_CHECK("block_resid_kernel");
      PF_CUDA(cudaMemcpyAsync(res.data(), S.res, nq * 8, cudaMemcpyDeviceToHost, S.st));
      clk.mark(5);
      PF_CUDA(cudaStreamSynchronize(S.st));
      S.rep.ms_check += clk.ms(4, 5);
      S.rep.checks++;
      double scale = 1.0;
      if (tol_relative) scale = std::max(std::fabs(th.front()), std::fabs(th.back()));
      bool ok = true;
      double rmax = 0.0;
      for (int i = 0; i < nq; ++i) {
        ok = ok && (res[i] <= tol * scale);
        rmax = std::max(rmax, res[i] / scale);
      }
      if (ok || last) {
        out.blocks = k;
        out.converged = ok || full;
        out.theta = th;
        out.idx = idx;
        out.resid = res;
        break;
      }
      // next check: every check_every blocks; earlier when the largest residual, extrapolated
      // geometrically from the last two checks, reaches tol sooner; where a check costs more than
      // half the block steps between two checks (the spectral-bounds Lanczos on H: a block step
      // is one SpMM with s = 4), at 3/4 of the extrapolated distance or at the budget.  The costs
      // are modelled from the sizes, never measured, so the steps taken do not depend on timing.
      int step = check_every;
      if (prev_k > 0 && rmax < prev_r && rmax > tol) {
        const double rate = std::log(rmax / prev_r) / (double)(k - prev_k);
        const double need = std::log(tol / rmax) / rate;
        step = std::max(1, std::min(check_every, (int)std::ceil(need) - 1));
        const double check_us = model_check_us(M, nq);
        const double block_us = model_block_us(S.H, s, K, k, op != OP_FILTER32);
        const int left = S.max_blocks - k;
        if (need > check_every && check_us > 0.5 * check_every * block_us && left > check_every)
          step = need >= left ? left : std::max(check_every, (int)(0.75 * need));
      }
      prev_k = k;
      prev_r = rmax;
      next_check = k + step;
    }
    if (last) {
      out.blocks = k;
      out.converged = false;
      break;
    }
  }
  return PF_OK;
}

// Dense copy of H (row-major D x D) from the CSR, FP64; A zeroed beforehand.
__global__ void csr_to_dense_kernel(int64_t D, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, double* A) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= D) return;
  for (int64_t j = rp[r]; j < rp[r + 1]; ++j) A[r * D + col[j]] += val[j];
}

// ||H z_c - w_c z_c|| for the columns z_c of Z (column-major, D x q), one CTA per column.
__global__ void csr_resid_kernel(int64_t D, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, const double* __restrict__ Z, const double* w,
                                 double* res) {
  __shared__ double sh[32];
  const int c = blockIdx.x;
  const double* z = Z + (int64_t)c * D;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < D; r += blockDim.x) {
    double h = 0.0;
    for (int64_t j = rp[r]; j < rp[r + 1]; ++j) h = fma(val[j], z[col[j]], h);
    const double d = h - w[c] * z[r];
    acc = fma(d, d, acc);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) res[c] = sqrt(acc);
}

// The extremes of a small H (D <= 400) from its dense form: one call of the H_L eigensolver (the
// thread-block-cluster tridiagonalisation) in place of a block Lanczos whose ~20 block steps and
// checks each cost launch latency (XXZ L = 10, D = 252: ~12 ms).  The residuals are computed from
// the CSR.
static pf_status spectral_bounds_dense(Ham* H, cudaStream_t st) {
  const int64_t D = H->D;
  DevBuf A, work, Z, wr;
  PF_TRY(A.alloc((size_t)D * D * 8, st));
  PF_CUDA(cudaMemsetAsync(A.p, 0, (size_t)D * D * 8, st));
  csr_to_dense_kernel<<<(unsigned)ceil_div(D, 128), 128, 0, st>>>(D, H->row_ptr, H->col, H->val, A.as<double>());
  PF_LAUNCH_CHECK("csr_to_dense_kernel");
  const size_t wb = eig_workspace_bytes((int)D, 2);
  PF_TRY(work.alloc(wb, st));
  PF_TRY(Z.alloc((size_t)D * 2 * 8, st));
  PF_TRY(wr.alloc(4 * 8, st));
  const int idx[2] = {0, (int)D - 1};
  double w[2] = {0, 0}, res[2] = {0, 0};
  PF_TRY(sym_eig_select(A.as<double>(), (int)D, (int)D, idx, 2, w, Z.as<double>(), (int)D, work.p, wb, st));
  PF_CUDA(cudaMemcpyAsync(wr.as<double>(), w, sizeof(w), cudaMemcpyHostToDevice, st));
  csr_resid_kernel<<<2, 256, 0, st>>>(D, H->row_ptr, H->col, H->val, Z.as<double>(), wr.as<double>(),
                                       wr.as<double>() + 2);
  PF_LAUNCH_CHECK("csr_resid_kernel");
  PF_CUDA(cudaMemcpyAsync(res, wr.as<double>() + 2, sizeof(res), cudaMemcpyDeviceToHost, st));
  PF_CUDA(cudaStreamSynchronize(st));
  H->emin = w[0];
  H->emax = w[1];
  H->rmin = res[0];
  H->rmax = res[1];
  return PF_OK;
}

static pf_status spectral_bounds_impl(Ham* H, double tol, cudaStream_t st) {
  if (tol <= 0) tol = 1e-10;
  if (H->D >= 4 && H->D <= 400) {
    PF_TRY(spectral_bounds_dense(H, st));
    H->hnorm = std::max(std::fabs(H->emin), std::fabs(H->emax));
    H->has_bounds = 1;
    const double de0 = 0.5 * (H->emax - H->emin);
    const double lo = H->emin - H->rmin - 1e-3 * de0;
    const double hi = H->emax + H->rmax + 1e-3 * de0;
    return set_rescale(H, 0.5 * (hi + lo), 0.5 * (hi - lo), st);
  }
  // Block width 4 (resolves extremal multiplicities up to 4).  When the whole space fits in
  // the Krylov budget (D <= 600), the width is a power of two dividing D, so the last block
  // completes the space and the extremes are then exact.
  int s = 4;
  while (s > 1 && 2 * s > H->D) s >>= 1;
  if (H->D <= 600)
    while (s > 1 && H->D % s != 0) s >>= 1;
  int max_blocks = (int)std::min<int64_t>(H->D / s, 600 / s);
  if (max_blocks < 1) max_blocks = 1;
  Solver S;
  PF_TRY(solver_init(S, H, s, max_blocks, 2, false, st));
  PF_TRY(start_block_raw(H->D, s, 0x5eedb0d5ull, blockp(S, 0), st));
  PF_TRY(chol_qr3(S, blockp(S, 0), blockp(S, 0)));
  LanczosResult R;
  PF_TRY(block_lanczos(S, OP_H, nullptr, 0, 0, 2, 2, tol, true, 5, 5, R));
  if (!R.converged) return PF_ENOTCONV;
  H->emin = R.theta.front();
  H->emax = R.theta.back();
  H->rmin = R.resid.front();
  H->rmax = R.resid.back();
  H->hnorm = std::max(std::fabs(H->emin), std::fabs(H->emax));
  H->has_bounds = 1;
  // padded interval (Lanczos extremes lie inside the spectrum)
  const double de0 = 0.5 * (H->emax - H->emin);
  const double lo = H->emin - H->rmin - 1e-3 * de0;
  const double hi = H->emax + H->rmax + 1e-3 * de0;
  return set_rescale(H, 0.5 * (hi + lo), 0.5 * (hi - lo), st);
}

// Guard factor (guard_factor, common.cuh): nev_g = ceil(g nev) Ritz pairs of P are converged and the
// degree K is chosen so that about nev_g eigenvalues lie above the cutoff.  The nev returned
// (nearest lambda) then have filter values P >~ sinc(2.655 / g) (0.55 at g = 1.5, 0.87 at 3),
// above the magnitude of the filter's negative sidelobe (~0.22), which is what the refinement must
// contract relative to them.  A larger guard lowers K (proportional to 1 / nev_g) faster than it
// grows the Krylov space (20.4 s + 1.7 nev_g): filter-dominated solves (D >= 100,000) take g = 3
// and need fewer steps in all; smaller ones, dominated by the Lanczos and Ritz work that grows
// with nev_g, keep g = 1.5.

static int expected_krylov_dim(int nev, int s, double eta) {
  return (int)std::ceil((20.427 * s + 1.696 * nev) * eta);
}

// H-space Rayleigh-Ritz on the blocked set U (nb blocks): U <- U Z, E = eig(U^T H U), residual norms.
static pf_status rayleigh_ritz_H(Solver& S, double* U, double* HU, int nb, std::vector<double>& E,
                                 std::vector<double>& res) {
  const int s = S.s;
  const int64_t D = S.D;
  const int q = nb * s;
  const Ham* H = S.H;
  for (int b = 0; b < nb; ++b) {
    const double* Ub = U + (int64_t)b * D * s;
    double* HUb = HU + (int64_t)b * D * s;
    PF_TRY(clenshaw_step_raw(D, H->row_ptr, H->col, H->val, PF_F64, s, Ub, Ub, nullptr, HUb, 0.0, 1.0, 0.0, S.st));
  }
  DevBuf G;
  PF_TRY(G.alloc((size_t)q * q * 8, S.st));
  PF_TRY((S.df ? gram_df : gram)(D, s, U, nb, HU, nb, G.as<double>(), S.gscr.as<double>(), S.gscr_elems, S.st));
  std::vector<int> idx(q);
  std::iota(idx.begin(), idx.end(), 0);
  E.assign(q, 0.0);
  DevBuf Zr, Cr, E_dev;
  PF_TRY(Zr.alloc((size_t)q * q * 8, S.st));
  PF_TRY(Cr.alloc((size_t)q * q * 8, S.st));
  size_t wb = eig_workspace_bytes(q, q);
  DevBuf ew;
  PF_TRY(ew.alloc(wb, S.st));
  PF_TRY(sym_eig_select(G.as<double>(), q, q, idx.data(), q, E.data(), Zr.as<double>(), q, ew.p, wb, S.st));
  // C row-major q x q from Zr (column-major)
  DevBuf perm;
  PF_TRY(perm.alloc(q * sizeof(int), S.st));
  PF_CUDA(cudaMemcpyAsync(perm.p, idx.data(), q * sizeof(int), cudaMemcpyHostToDevice, S.st));
  z_to_rowmajor_kernel<<<(unsigned)ceil_div((int64_t)q * q, 256), 256, 0, S.st>>>(Zr.as<double>(), q, q, q,
                                                                                   perm.as<int>(), Cr.as<double>(), q);
  PF_LAUNCH_CHECK("z_to_rowmajor_kernel");
  // U2 = U C into HU's storage, then copy back; HU recomputed from U2
  for (int b = 0; b < nb; ++b)
    PF_TRY((S.df ? tsgemm_df : tsgemm)(D, s, U, nb, Cr.as<double>() + b * s, q, HU + (int64_t)b * D * s, 1,
                  1.0, 0.0, S.st));
  PF_CUDA(cudaMemcpyAsync(U, HU, (size_t)nb * D * s * 8, cudaMemcpyDeviceToDevice, S.st));
  for (int b = 0; b < nb; ++b) {
    const double* Ub = U + (int64_t)b * D * s;
    double* HUb = HU + (int64_t)b * D * s;
    PF_TRY(clenshaw_step_raw(D, H->row_ptr, H->col, H->val, PF_F64, s, Ub, Ub, nullptr, HUb, 0.0, 1.0, 0.0, S.st));
  }
  PF_TRY(E_dev.alloc(q * 8, S.st));
  PF_CUDA(cudaMemcpyAsync(E_dev.p, E.data(), q * 8, cudaMemcpyHostToDevice, S.st));
  DevBuf rn;
  PF_TRY(rn.alloc(q * 8, S.st));
  PF_TRY(colnorms(D, s, HU, U, E_dev.as<double>(), nb, rn.as<double>(), S.gscr.as<double>(),
                  S.gscr_elems, S.st));
  res.assign(q, 0.0);
  PF_CUDA(cudaMemcpyAsync(res.data(), rn.p, q * 8, cudaMemcpyDeviceToHost, S.st));
  PF_CUDA(cudaStreamSynchronize(S.st));
  return PF_OK;
}

// Orthonormalise a blocked set (nb blocks) with two Cholesky-QR passes on the whole set.
static pf_status orthonormalise_set(Solver& S, double* U, double* T, int nb) {
  const int s = S.s;
  const int q = nb * s;
  const int64_t D = S.D;
  DevBuf G, R, Ri, st;
  PF_TRY(G.alloc((size_t)q * q * 8, S.st));
  PF_TRY(R.alloc((size_t)q * q * 8, S.st));
  PF_TRY(Ri.alloc((size_t)q * q * 8, S.st));
  PF_TRY(st.alloc(16, S.st));
  const double u = 1.1102230246251565e-16;
  for (int pass = 0; pass < 2; ++pass) {
    PF_TRY((S.df ? gram_df : gram)(D, s, U, nb, U, nb, G.as<double>(), S.gscr.as<double>(), S.gscr_elems, S.st));
    const double shift = pass == 0 ? 11.0 * ((double)D * q + (double)q * (q + 1)) * u : 0.0;
    PF_TRY(small_chol_inv(G.as<double>(), q, shift, R.as<double>(), Ri.as<double>(), st.as<int>(), S.st));
    for (int b = 0; b < nb; ++b)
      PF_TRY((S.df ? tsgemm_df : tsgemm)(D, s, U, nb, Ri.as<double>() + b * s, q, T + (int64_t)b * D * s, 1, 1.0,
                    0.0, S.st));
    PF_CUDA(cudaMemcpyAsync(U, T, (size_t)nb * D * s * 8, cudaMemcpyDeviceToDevice, S.st));
    int bad = 0;
    PF_CUDA(cudaMemcpyAsync(&bad, st.p, sizeof(int), cudaMemcpyDeviceToHost, S.st));
    PF_CUDA(cudaStreamSynchronize(S.st));
    if (bad) return PF_EBREAKDOWN;
  }
  return PF_OK;
}

static std::vector<int> nearest_sel(const std::vector<double>& E, double lam, int nev) {
  std::vector<int> o(E.size());
  std::iota(o.begin(), o.end(), 0);
  std::sort(o.begin(), o.end(), [&](int a, int b) {
    double da = std::fabs(E[a] - lam), db = std::fabs(E[b] - lam);
    if (da != db) return da < db;
    return E[a] < E[b];
  });
  o.resize(std::min<size_t>(nev, o.size()));
  std::sort(o.begin(), o.end(), [&](int a, int b) { return E[a] < E[b]; });
  return o;
}

// ------------------------------------------------------------------ block-width autotuner
// The block width s trades matrix reuse against Krylov size: one Clenshaw step over a D x s
// block costs t(s) (measured here: 8 steps of the step kernel on scratch blocks, per
// candidate), and the Krylov space needs about expectedkrylovdim(nev_g, s, 1) / s blocks of
// K+1 steps (Sec. 5.5: (20.427 s + 1.696 nev_g) / s).  The choice minimises the predicted
// filter time of the Lanczos stage, blocks(s) x t(s), over s in {8, 16, 32, 64} with s not above
// the padded guard count.  Measured once per (device, D, nnz, precision).
namespace {
struct BlockKey {
  int dev, prec;
  int64_t D, nnz;
  bool operator<(const BlockKey& o) const { return std::tie(dev, prec, D, nnz) < std::tie(o.dev, o.prec, o.D, o.nnz); }
};
std::mutex g_block_mu;
std::map<BlockKey, std::array<double, 4>> g_block_us;
}  // namespace

static const int kBlockCand[4] = {8, 16, 32, 64};

static pf_status measure_block_steps(const Ham* H, int prec, cudaStream_t st, std::array<double, 4>& us) {
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  const BlockKey key{dev, prec, H->D, H->nnz};
  {
    std::lock_guard<std::mutex> lock(g_block_mu);
    auto f = g_block_us.find(key);
    if (f != g_block_us.end()) {
      us = f->second;
      return PF_OK;
    }
  }
  const size_t w = prec_bytes(prec);
  const size_t blk = (size_t)H->D * 64 * w;
  DevBuf buf;
  PF_TRY(buf.alloc(3 * blk, st));
  PF_CUDA(cudaMemsetAsync(buf.p, 0, 3 * blk, st));
  unsigned char* b = buf.as<unsigned char>();
  cudaEvent_t e0, e1;
  PF_CUDA(cudaEventCreate(&e0));
  PF_CUDA(cudaEventCreate(&e1));
  pf_status rc = PF_OK;
  for (int c = 0; c < 4 && rc == PF_OK; ++c) {
    const int sc = kBlockCand[c];
    auto step = [&] {
      return ham_step(H, prec, sc, b, b + blk, b + 2 * blk, b + 2 * blk, 0.5, 2.0, 1.0, st);
    };
    rc = step();   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 8 && rc == PF_OK; ++r) rc = step();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    us[c] = 1e3 * ms / 8;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  PF_TRY(rc);
  std::lock_guard<std::mutex> lock(g_block_mu);
  g_block_us[key] = us;
  return PF_OK;
}

static int expected_krylov_dim(int nev, int s, double eta);

static pf_status autotune_block(const Ham* H, int prec, int nev, cudaStream_t st, int* s_out, double* us_out,
                                double* cost_out, int refine_prec = PF_F64) {
  std::array<double, 4> us, us64;
  PF_TRY(measure_block_steps(H, prec, st, us));
  if (prec == PF_F32) PF_TRY(measure_block_steps(H, refine_prec, st, us64));
  const int nev_g = std::max(nev, (int)std::ceil(guard_factor((double)H->D) * nev));
  double best = 0;
  int bs = 0;
  for (int c = 0; c < 4; ++c) {
    const int sc = kBlockCand[c];
    if (sc > 8 && sc > nev_g) break;                        // wider than the guard: no gain
    if ((int64_t)sc * 2 > H->D) break;
    const double blocks = std::ceil(expected_krylov_dim(nev_g, sc, 1.0) / (double)sc);
    double cost = blocks * us[c];
    // FP32 path: refinement of the guard set, ~1.3 passes at degree 0.7 K on average
    if (prec == PF_F32) cost += 1.3 * 0.7 * std::ceil(nev_g / (double)sc) * us64[c];
    if (cost_out) cost_out[c] = cost;
    if (bs == 0 || cost < best) {
      best = cost;
      bs = sc;
    }
  }
  if (us_out)
    for (int c = 0; c < 4; ++c) us_out[c] = us[c];
  *s_out = bs ? bs : 8;
  return PF_OK;
}

// ------------------------------------------------------------------ resumable solve
// One POLFED solve as a resumable task.  The filter applications the task needs next are
// listed in `pending`; an executor runs the pending applications of all active tasks
// (items with the same precision and block width share one sweep) and then calls
// after_filter(), which does the task's orthogonalisation, QR, checks, extraction or
// refinement work and lists the next applications.  pf_polfed_solve runs one task,
// pf_polfed_solve_batch and the server run many.  The filter kernels compute every row with
// the same operation order in all three paths, so a task's results do not depend on
// which other tasks share its sweeps.
struct Task {
  enum Phase { LANCZOS = 0, REFINE = 1, DONE = 2 };
  Ham* H = nullptr;
  cudaStream_t st = 0;
  pf_solve_opts o;
  int nev = 0, K = 0, s = 0, nev_g = 0, max_blocks = 0, check_first = 0, check_every = 0;
  // convergence checks: the next block step at which one runs, and the previous check's block and
  // largest residual (for the extrapolated cadence)
  int next_check = 0, prev_check_k = 0;
  double prev_check_r = 0;
  int qb = 0, qpad = 0, q_reserve = 0;
  bool f32 = false;
  double tol = 0, res_tol = 0, lam = 0, lam_t = 0, hnorm = 0;
  Solver S;
  DevBuf coeff_dev, coeffr_dev;
  std::vector<double> coeffs, coeffs_r;
  Phase phase = LANCZOS;
  int k = 0;                      // Krylov blocks completed
  LanczosResult R;
  int nb = 0, nb_total = 0, passes = 0, max_pass = 0, Kr = 0, Lb = 0, na = 0;
  double prev = 0, a0 = 0;
  DevBuf U, HU, aux64;
  DevBuf corr_small;   // correction form, per block: C = U^T H~ U, P(theta), theta
  bool corr_fits = false;   // the gamma tables fit in the (then idle) Krylov basis
  std::vector<double> E, res;
  std::vector<int> sel;
  std::vector<FilterItem> pending;
  pf_status status = PF_OK;
  PhaseClock* clk = nullptr;
  // Captured filter applications, used when an asynchronous executor drives the task: the
  // Lanczos filter reads a fixed input block (Vin, FP64 path) so one graph serves every step.
  bool captured = false;
  DevBuf Vin;
  FilterGraph g_lanczos;
  std::vector<std::unique_ptr<FilterGraph>> g_refine;
  cudaEvent_t t_begin = nullptr, t_end = nullptr;

  Task() { memset(&o, 0, sizeof(o)); }
  Task(const Task&) = delete;
  Task& operator=(const Task&) = delete;
  ~Task() {
    delete clk;
    if (t_begin) cudaEventDestroy(t_begin);
    if (t_end) cudaEventDestroy(t_end);
  }

  // arithmetic of the refinement filter in the direct form (PF_DF64 or PF_F64)
  int refine_prec() const { return o.refine_precision; }
  // Gram-Schmidt passes and Ritz-vector assembly in pair-float arithmetic (orth_precision)
  bool orth_df() const { return o.orth_precision == PF_DF64 || (o.orth_precision == 0 && f32); }
  // refinement passes in the residual-correction form: asked for, or the default with the FP64
  // refinement arithmetic (an explicit pair-float request keeps the direct form); needs K >= 2
  bool corr_form() const {
    const bool want = o.refine_form == PF_REFINE_CORRECTION || (o.refine_form == 0 && o.refine_precision == PF_F64);
    return f32 && want && Kr >= 2 && corr_fits;
  }
  // The per-block gamma tables (FP32, up to K rows of s) live in the Krylov basis, which the
  // refinement no longer reads once the Ritz vectors are extracted.
  float* corr_gamma(int b) const { return reinterpret_cast<float*>(S.V.as<double>()) + (int64_t)b * K * s; }

  double max_res() const {
    double m = 0;
    for (int j : sel) m = std::max(m, res[j]);
    return m;
  }

  // Validates the request, allocates the resident state, draws and orthonormalises the
  // start block and lists the first filter application.
  pf_status init(Ham* Hh, double target_eps, int nev_, int K_, const pf_solve_opts* o_in, cudaStream_t stream) {
    pf_default_opts(&o);
    if (o_in) o = *o_in;
    H = Hh;
    st = stream;
    nev = nev_;
    K = K_;
    if (!H) return PF_EINVAL;
    if (!H->has_rescale) return PF_ESTATE;
    if (!o.use_abs_target && !H->has_bounds) return PF_ESTATE;
    if (nev < 1 || nev > H->D || K < 1) return PF_EINVAL;
    if (!o.use_abs_target && !(target_eps >= 0.0 && target_eps <= 1.0)) return PF_EINVAL;
    if (o.precision != PF_F64 && o.precision != PF_F32) return PF_EINVAL;
    if (o.refine_precision != PF_F64 && o.refine_precision != PF_DF64) return PF_EINVAL;
    if (o.refine_form != 0 && o.refine_form != PF_REFINE_DIRECT && o.refine_form != PF_REFINE_CORRECTION)
      return PF_EINVAL;
    if (o.orth_precision != 0 && o.orth_precision != PF_F64 && o.orth_precision != PF_DF64) return PF_EINVAL;
    if (o.block < 0) {   // the autotuner picks the block width
      if (!H->has_rescale) return PF_ESTATE;
      PF_TRY(autotune_block(H, o.precision, nev, stream, &s, nullptr, nullptr, refine_prec()));
      o.block = s;
    }
    s = o.block > 0 ? o.block : 32;
    if (!(s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32 || s == 64)) return PF_EINVAL;
    f32 = o.precision == PF_F32;
    const double eta = o.eta > 0 ? o.eta : 1.5;
    tol = f32 ? (o.tol_f32 > 0 ? o.tol_f32 : 1e-7) : (o.tol > 0 ? o.tol : 1e-10);
    res_tol = o.res_tol > 0 ? o.res_tol : 1e-9;
    nev_g = o.nev_guard > 0 ? o.nev_guard : (int)std::ceil(guard_factor((double)H->D) * nev);
    nev_g = std::max(nev_g, nev);
    if (nev_g > H->D) nev_g = (int)H->D;
    const int Mmax = (int)std::min<int64_t>(expected_krylov_dim(nev_g, s, eta), H->D);
    max_blocks = o.max_blocks > 0 ? o.max_blocks : std::max(2, Mmax / s);
    if ((int64_t)max_blocks * s > H->D) max_blocks = (int)(H->D / s);
    if (max_blocks < 1 || (int64_t)max_blocks * s < (int64_t)((nev_g + s - 1) / s) * s) return PF_EINVAL;
    const int m_est = std::max(1, (int)std::ceil(expected_krylov_dim(nev_g, s, 1.0) / (double)s));
    check_first = o.check_first > 0 ? o.check_first : std::max(1, (int)std::ceil(0.5 * m_est));
    check_every = o.check_every > 0 ? o.check_every : std::max(1, (int)std::ceil(0.1 * m_est));
    next_check = check_first;
    qb = (nev_g + s - 1) / s;      // Ritz blocks extracted
    qpad = qb * s;
    // extra Ritz vectors kept for the refinement set
    q_reserve = f32 ? (o.refine_reserve < 0 ? 0 : (o.refine_reserve == 0 ? 2 : o.refine_reserve)) * s : 0;
    lam = o.use_abs_target ? o.target_abs : H->emin + target_eps * (H->emax - H->emin);
    lam_t = (lam - H->Ec) / H->dE;
    if (!(lam_t > -1.0 && lam_t < 1.0)) return PF_EINVAL;
    PF_CUDA(cudaEventCreate(&t_begin));
    PF_CUDA(cudaEventCreate(&t_end));
    PF_CUDA(cudaEventRecord(t_begin, st));
    clk = new PhaseClock(st);
    PF_TRY(solver_init(S, H, s, max_blocks, std::max(qpad + q_reserve, nev_g), f32, st));
    S.df = orth_df();
    coeffs.resize(K + 1);
    PF_TRY(filter_coefficients_dev(lam_t, K, coeffs.data(), st));
    PF_TRY(coeff_dev.alloc((size_t)(K + 1) * 8, st));
    PF_CUDA(cudaMemcpyAsync(coeff_dev.p, coeffs.data(), (size_t)(K + 1) * 8, cudaMemcpyHostToDevice, st));
    S.rep.K = K;
    S.rep.nev_guard = nev_g;
    S.rep.lambda = lam;
    S.rep.lambda_t = lam_t;
    S.rep.emin = H->emin;
    S.rep.emax = H->emax;
    S.rep.Ec = H->Ec;
    S.rep.dE = H->dE;
    hnorm = H->has_bounds ? H->hnorm : std::max(std::fabs(H->Ec - H->dE), std::fabs(H->Ec + H->dE));
    S.rep.hnorm = hnorm;
    PF_TRY(start_block_raw(H->D, s, o.seed, blockp(S, 0), st));
    PF_TRY(chol_qr3(S, blockp(S, 0), blockp(S, 0)));
    return issue_lanczos_filter();
  }

  // W = P(H~) V_k: FP64 directly on the basis block, or FP32 on a converted copy.
  pf_status issue_lanczos_filter() {
    double* Vk = blockp(S, k);
    FilterItem it;
    it.H = H;
    it.owner = this;
    it.s = s;
    it.coeffs_host = coeffs.data();
    it.coeffs_dev = coeff_dev.as<double>();
    it.K = K;
    it.aux0 = S.aux0.p;
    it.aux1 = S.aux1.p;
    if (f32) {
      PF_TRY(convert_d2f(Vk, S.V32.as<float>(), S.D * s, st));
      it.prec = PF_F32;
      it.V = S.V32.p;
      it.W = S.W32.p;
      S.rep.filter_steps_f32 += K + 1;
    } else {
      it.prec = PF_F64;
      it.V = Vk;
      it.W = S.W.p;
      S.rep.filter_steps_f64 += K + 1;
      if (captured) {
        if (!Vin.p) PF_TRY(Vin.alloc((size_t)S.D * s * 8, st));
        PF_CUDA(cudaMemcpyAsync(Vin.p, Vk, (size_t)S.D * s * 8, cudaMemcpyDeviceToDevice, st));
        it.V = Vin.p;
      }
    }
    it.graph = &g_lanczos;
    clk->mark(0);
    pending.assign(1, it);
    return PF_OK;
  }

  pf_status after_filter() {
    pending.clear();
    if (phase == LANCZOS) return lanczos_post();
    if (phase == REFINE) return refine_post();
    return PF_OK;
  }

  // The rest of block step k after W = P V_k: A_k, two Gram-Schmidt passes against the whole
  // basis, shifted Cholesky QR, H_L, and the periodic convergence check.
  pf_status lanczos_post() {
    const int64_t D = S.D;
    double* W = S.W.as<double>();
    double* Vk = blockp(S, k);
    clk->mark(1);
    if (f32) PF_TRY(convert_f2d(S.W32.as<float>(), W, D * s, st));
    PF_TRY(gram(D, s, Vk, 1, W, 1, S.Ab, S.gscr.as<double>(), S.gscr_elems, st));
    hl_store_kernel<<<1, 256, 0, st>>>(S.HL.as<double>(), S.Mcap, k, s, S.Ab, nullptr);
    PF_LAUNCH_CHECK("hl_store_kernel");
    for (int pass = 0; pass < 2; ++pass) {
      if (orth_df() && (s == 16 || s == 32 || s == 64)) {
        // W split into float pairs once (into tmp, free until the QR), shared by every basis block
        float2* W2 = reinterpret_cast<float2*>(S.tmp.p);
        PF_TRY(convert_d2df(W, W2, D * s, st));
        PF_TRY(gram_df_ysplit(D, s, S.V.as<double>(), k + 1, W2, 1, S.Cg.as<double>(), S.gscr.as<double>(),
                              S.gscr_elems, st));
        PF_TRY(tsgemm_df(D, s, S.V.as<double>(), k + 1, S.Cg.as<double>(), s, W, 1, -1.0, 1.0, st));
      } else if (orth_df()) {
        PF_TRY(gram_df(D, s, S.V.as<double>(), k + 1, W, 1, S.Cg.as<double>(), S.gscr.as<double>(), S.gscr_elems, st));
        PF_TRY(tsgemm_df(D, s, S.V.as<double>(), k + 1, S.Cg.as<double>(), s, W, 1, -1.0, 1.0, st));
      } else {
        PF_TRY(gram(D, s, S.V.as<double>(), k + 1, W, 1, S.Cg.as<double>(), S.gscr.as<double>(), S.gscr_elems, st));
        PF_TRY(tsgemm(D, s, S.V.as<double>(), k + 1, S.Cg.as<double>(), s, W, 1, -1.0, 1.0, st));
      }
    }
    clk->mark(2);
    // full: the basis spans the whole space, so B_{k+1} = 0 exactly.  cap: no room for
    // another block; B_{k+1} comes from the Cholesky factor of W^T W alone (enough for
    // ||B tau||), and the iteration stops.
    const bool full = (int64_t)(k + 1) * s >= D;
    const bool cap = (int64_t)(k + 2) * s > D;
    if (full) {
      PF_CUDA(cudaMemsetAsync(S.Bb, 0, (size_t)s * s * 8, st));
    } else if (cap) {
      const double u = 1.1102230246251565e-16;
      PF_TRY(gram(D, s, W, 1, W, 1, S.Gb, S.gscr.as<double>(), S.gscr_elems, st));
      PF_TRY(small_chol_inv(S.Gb, s, 11.0 * ((double)D * s + (double)s * (s + 1)) * u, S.Bb, S.Rib, S.stat, st));
    } else {
      PF_TRY(chol_qr3(S, W, blockp(S, k + 1)));
    }
    hl_store_kernel<<<1, 256, 0, st>>>(S.HL.as<double>(), S.Mcap, k, s, nullptr, S.Bb);
    PF_LAUNCH_CHECK("hl_store_kernel");
    clk->mark(3);
    (f32 ? S.rep.ms_filter_f32 : S.rep.ms_filter_f64) += clk->ms(0, 1);
    S.rep.ms_orth += clk->ms(1, 2);
    S.rep.ms_qr += clk->ms(2, 3);
    ++k;
    const int M = k * s;
    const bool last = (k + 1 > S.max_blocks) || full || cap;
    const bool enough = M >= nev_g && M >= qpad;
    const bool at_check = k >= next_check || last;
    if (enough && at_check) {
      std::vector<int> idx;
      for (int i = M - nev_g; i < M; ++i) idx.push_back(i);
      const int nq = (int)idx.size();
      std::vector<double> th(nq), rr(nq);
      clk->mark(4);
      PF_TRY(sym_eig_select(S.HL.as<double>(), S.Mcap, M, idx.data(), nq, th.data(), S.Z.as<double>(), M, S.eigw.p,
                            S.eig_bytes, st));
      block_resid_kernel<<<(unsigned)ceil_div(nq, 64), 64, 0, st>>>(S.Bb, s, S.Z.as<double>(), M, M, nq, S.res);
      PF_LAUNCH_CHECK("block_resid_kernel");
      PF_CUDA(cudaMemcpyAsync(rr.data(), S.res, nq * 8, cudaMemcpyDeviceToHost, st));
      clk->mark(5);
      PF_CUDA(cudaStreamSynchronize(st));
      S.rep.ms_check += clk->ms(4, 5);
      S.rep.checks++;
      bool ok = true;
      double rmax = 0;
      for (int i = 0; i < nq; ++i) {
        ok = ok && (rr[i] <= tol);
        rmax = std::max(rmax, rr[i]);
      }
      // Next check: every check_every block steps; with the default cadence, earlier when the
      // largest residual, extrapolated geometrically from the last two checks, reaches tol sooner
      // (one step before the predicted block).  A block step at L = 20 costs ~4x a check.  Where a
      // check costs more than half the block steps between two checks (small sectors, many
      // eigenpairs: XXZ L = 16, s = 16, nev = 200 checks at n ~ 400-1250 for 10-30 ms against ~1 ms
      // per block), the next check moves to 3/4 of the extrapolated distance, or straight to the
      // Krylov budget when the extrapolation lies beyond it.  Both costs are modelled from the
      // sizes (model_check_us, model_block_us), never measured: the Krylov dimension a solve stops
      // at, and so its result, must not depend on what else runs on the GPU.
      int step = check_every;
      if (o.check_every <= 0 && prev_check_k > 0 && rmax < prev_check_r && rmax > tol) {
        const double rate = std::log(rmax / prev_check_r) / (double)(k - prev_check_k);
        const double need = std::log(tol / rmax) / rate;
        step = std::max(1, std::min(check_every, (int)std::ceil(need) - 1));
        const int left = S.max_blocks - k;
        const double check_us = model_check_us(M, nq);
        const double block_us = model_block_us(H, s, K, k, !f32);
        if (need > check_every && check_us > 0.5 * check_every * block_us && left > check_every)
          step = need >= left ? left : std::max(check_every, (int)(0.75 * need));
      }
      prev_check_k = k;
      prev_check_r = rmax;
      next_check = k + step;
      if (ok || last) {
        R.blocks = k;
        R.converged = ok || full;
        R.theta = th;
        R.idx = idx;
        R.resid = rr;
        return extract();
      }
    }
    if (last) {
      R.blocks = k;
      R.converged = false;
      return PF_ENOTCONV;
    }
    return issue_lanczos_filter();
  }

  // Ritz vectors for the largest theta: qb blocks (the nev_g checked, padded to whole blocks)
  // and, for the FP32 filter, up to two reserve blocks that join the refinement set when it
  // stalls; Rayleigh-Ritz in H; then refinement or done.
  pf_status extract() {
    const int M = R.blocks * s;
    S.rep.blocks = R.blocks;
    S.rep.krylov_dim = M;
    clk->mark(0);
    nb_total = std::min(qb + q_reserve / s, M / s);
    const int qtot = nb_total * s;
    std::vector<int> idx;
    for (int i = M - qtot; i < M; ++i) idx.push_back(i);
    std::vector<double> th(qtot);
    PF_TRY(sym_eig_select(S.HL.as<double>(), S.Mcap, M, idx.data(), qtot, th.data(), S.Z.as<double>(), M, S.eigw.p,
                          S.eig_bytes, st));
    // C (M x qtot row-major): columns are the Ritz coefficient vectors, largest theta first
    DevBuf perm;
    std::vector<int> pv(qtot);
    for (int c = 0; c < qtot; ++c) pv[c] = qtot - 1 - c;
    PF_TRY(perm.alloc(qtot * sizeof(int), st));
    PF_CUDA(cudaMemcpyAsync(perm.p, pv.data(), qtot * sizeof(int), cudaMemcpyHostToDevice, st));
    z_to_rowmajor_kernel<<<(unsigned)ceil_div((int64_t)M * qtot, 256), 256, 0, st>>>(
        S.Z.as<double>(), M, M, qtot, perm.as<int>(), S.Cg.as<double>(), qtot);
    PF_LAUNCH_CHECK("z_to_rowmajor_kernel");
    PF_TRY(U.alloc((size_t)nb_total * H->D * s * 8, st));
    PF_TRY(HU.alloc((size_t)nb_total * H->D * s * 8, st));
    for (int b = 0; b < nb_total; ++b)
      PF_TRY((orth_df() ? tsgemm_df : tsgemm)(H->D, s, S.V.as<double>(), R.blocks, S.Cg.as<double>() + b * s, qtot,
                                              U.as<double>() + (int64_t)b * H->D * s, 1, 1.0, 0.0, st));
    nb = qb;   // active Ritz blocks; blocks nb..nb_total-1 of U hold the reserve
    PF_TRY(rayleigh_ritz_H(S, U.as<double>(), HU.as<double>(), qb, E, res));
    sel = nearest_sel(E, lam, nev);
    clk->mark(1);
    S.rep.ms_extract = clk->ms(0, 1);
    S.rep.max_residual_unrefined = max_res();
    // FP64 refinement for the FP32 filter: subspace iteration U <- (P(H~) + c I) U on the
    // active blocks, Cholesky QR, Rayleigh-Ritz in H.  An error component on eigenvalue k
    // shrinks by |P_k + c| / (P_j + c) per pass for wanted pair j.  The first pass is
    // unshifted (c = 0), which removes the far bulk (P ~ 0) fastest.  What remains after it
    // sits where |P| is comparable to the edge pairs' P (~0.6): the filter's negative sidelobe
    // (minimum ~ -0.22) and the positive values just outside the set (second peak ~0.13).
    // Later passes use c = 0.05 (option refine_shift), which makes the two contraction
    // factors about equal, (0.22 - c)/(0.6 + c) ~ (0.13 + c)/(0.6 + c) ~ 0.27, against 0.36
    // unshifted; the far bulk, already gone, then shrinks only by c/(0.6 + c).  A pass that
    // gains less than 10x also adds one reserve block to the set.
    max_pass = o.refine_passes < 0 ? 0 : (o.refine_passes == 0 ? 8 : o.refine_passes);
    // degree of the refinement filter: 0.7 K by default when K >= 1000 (measured at L=20,
    // W = 1, 3, 5: the passes and blocks filtered stay the same as with K, and each pass costs
    // 30 % less; 0.55 K needs extra passes).  Low-degree filters (small sectors, targets near
    // the spectral edge) keep K: there the wider lobe let a reserve block bring in a spurious
    // pair (XXZ L=16, nev=100, K=114 stalled at 0.06 ||H||, and converges with K).
    Kr = o.refine_K > 0 ? o.refine_K : (K >= 1000 ? (int)(0.7 * K) : K);
    if (f32 && max_res() > res_tol * hnorm && max_pass > 0) {
      coeffs_r.resize(Kr + 1);
      PF_TRY(filter_coefficients_dev(lam_t, Kr, coeffs_r.data(), st));
      a0 = coeffs_r[0];
      PF_TRY(coeffr_dev.alloc((size_t)(std::max(Kr, K) + 1) * 8, st));
      PF_TRY(aux64.alloc((size_t)2 * nb_total * H->D * s * 8, st));
      // room for the largest degree a pass can take (K after a stall) in the basis' bytes
      corr_fits = Kr <= K && (size_t)nb_total * K * s * sizeof(float) <= S.V.bytes;
      if (corr_form()) PF_TRY(corr_small.alloc((size_t)nb_total * (s * s + 2 * s) * sizeof(double), st));
      prev = max_res();
      phase = REFINE;
      if (o.refine_full_set && nb < nb_total) {   // the reserve joins the set now
        nb = nb_total;
        res.resize(qb * s);                       // reserve columns have no residual yet
      }
      return issue_refine_filter();
    }
    return finish();
  }

  // Locking: returned pairs already within refine_lock x the tolerance (other pairs of the set within
  // refine_guard_lock x the tolerance) stay in the set but are not filtered; they move to the
  // leading blocks (rounded down to whole blocks by keeping the worst of them active).
  // Columns without a residual yet (a reserve block just added) are active.  Each active block
  // is one filter item with its own auxiliary pair.
  pf_status issue_refine_filter() {
    const double c_shift = o.refine_shift == 0.0 ? 0.05 : (o.refine_shift < 0.0 ? 0.0 : o.refine_shift);
    coeffs_r[0] = passes > 0 ? a0 + c_shift : a0;
    const int rprec = refine_prec();
    const bool corr = corr_form();
    {
      std::vector<double> tab(Kr + 1);   // pageable: consumed when the copy call returns
      coeff_table_host(corr ? PF_F64 : rprec, coeffs_r.data(), Kr + 1, tab.data());
      PF_CUDA(cudaMemcpyAsync(coeffr_dev.p, tab.data(), (size_t)(Kr + 1) * 8, cudaMemcpyHostToDevice, st));
    }
    const int q = nb * s;
    const int64_t DS = H->D * s;
    double* Ud = U.as<double>();
    double* HUd = HU.as<double>();
    std::vector<char> is_sel(q, 0);
    for (int j : sel) is_sel[j] = 1;
    // Guard and reserve pairs only span the buffer the returned pairs converge against; once
    // accurate to a few times the tolerance they stop being filtered too (a later pass unlocks
    // any whose residual grows again).
    const double glock = o.refine_guard_lock == 0.0 ? 10.0 : o.refine_guard_lock;
    // returned pairs lock once within rlock x the tolerance (0.9 by default: at 0.5, XXZ L=20
    // W=5 filtered 4 of 5 blocks again in its second pass, at 0.9 two, 2 s less per solve)
    const double rlock = o.refine_lock > 0.0 ? std::min(o.refine_lock, 1.0) : 0.9;
    std::vector<int> locked, active;
    for (int c = 0; c < q; ++c) {
      const bool have = c < (int)res.size();
      const bool lock_sel = have && is_sel[c] && res[c] <= rlock * res_tol * hnorm;
      const bool lock_guard = have && !is_sel[c] && glock > 0 && res[c] <= glock * res_tol * hnorm;
      if (lock_sel || lock_guard) locked.push_back(c);
      else active.push_back(c);
    }
    std::sort(locked.begin(), locked.end(), [&](int x, int y) { return res[x] < res[y]; });
    while (active.size() % s != 0) {
      active.push_back(locked.back());
      locked.pop_back();
    }
    Lb = (int)locked.size() / s;
    na = nb - Lb;
    if (Lb > 0) {
      std::vector<int> order(locked);
      order.insert(order.end(), active.begin(), active.end());
      DevBuf pd;
      PF_TRY(pd.alloc(q * sizeof(int), st));
      PF_CUDA(cudaMemcpyAsync(pd.p, order.data(), q * sizeof(int), cudaMemcpyHostToDevice, st));
      permute_cols_kernel<<<(unsigned)ceil_div(H->D * q, 256), 256, 0, st>>>(H->D, s, Ud, pd.as<int>(), q, HUd);
      PF_LAUNCH_CHECK("permute_cols_kernel");
      PF_CUDA(cudaMemcpyAsync(Ud, HUd, (size_t)q * H->D * 8, cudaMemcpyDeviceToDevice, st));
      PF_CUDA(cudaStreamSynchronize(st));
    }
    clk->mark(2);
    pending.clear();
    // Pair-float filter: the active blocks are converted into the HU blocks, which the filter
    // reads as V and which hold its FP64 result after refine_post converts W back; W is
    // written over the active U blocks, which are only scratch until the set is rebuilt.
    if (corr) return issue_refine_correction();
    const bool pair = rprec == PF_DF64;
    if (pair && na > 0)
      PF_TRY(convert_d2df(Ud + (int64_t)Lb * DS, reinterpret_cast<float2*>(HUd + (int64_t)Lb * DS), na * DS, st));
    for (int b = Lb; b < nb; ++b) {
      FilterItem it;
      it.H = H;
      it.owner = this;
      it.prec = rprec;
      it.s = s;
      it.V = pair ? (const void*)(HUd + (int64_t)b * DS) : (const void*)(Ud + (int64_t)b * DS);
      it.W = pair ? (void*)(Ud + (int64_t)b * DS) : (void*)(HUd + (int64_t)b * DS);
      it.coeffs_host = coeffs_r.data();
      it.coeffs_dev = coeffr_dev.as<double>();
      it.K = Kr;
      it.aux0 = aux64.as<double>() + (int64_t)(2 * b) * DS;
      it.aux1 = aux64.as<double>() + (int64_t)(2 * b + 1) * DS;
      while ((int)g_refine.size() <= b) g_refine.emplace_back(new FilterGraph());
      it.graph = g_refine[b].get();
      pending.push_back(it);
      S.rep.filter_steps_f64 += Kr + 1;
    }
    return PF_OK;
  }

  // Correction form: per active block, H~ U (FP64 step), C = U^T H~ U, the gamma table and
  // P(theta) (corr_table_kernel), r = H~ U - theta U in FP32, then the FP32 d recurrence of degree
  // Kr - 1 on r with per-column coefficients, written to the block's FP32 slots of aux64: r, dW,
  // and the two recurrence auxiliaries (the 2 D s doubles of a block hold 4 D s floats).
  pf_status issue_refine_correction() {
    const int64_t DS = H->D * s;
    double* Ud = U.as<double>();
    double* HUd = HU.as<double>();
    for (int b = Lb; b < nb; ++b) {
      const double* Ub = Ud + (int64_t)b * DS;
      double* HUb = HUd + (int64_t)b * DS;
      double* Cb = corr_small.as<double>() + (int64_t)b * (s * s + 2 * s);
      float* gam = corr_gamma(b);
      float* f = reinterpret_cast<float*>(aux64.as<double>() + (int64_t)(2 * b) * DS);
      PF_TRY(ham_step(H, PF_F64, s, Ub, Ub, nullptr, HUb, 0.0, 1.0, 0.0, st));
      PF_TRY(gram(H->D, s, Ub, 1, HUb, 1, Cb, S.gscr.as<double>(), S.gscr_elems, st));
      corr_table_kernel<<<1, 64, 0, st>>>(coeffr_dev.as<double>(), Kr, Cb, s, gam, Cb + s * s, Cb + s * s + s);
      PF_LAUNCH_CHECK("corr_table_kernel");
      corr_resid_kernel<<<(unsigned)ceil_div(DS, 256), 256, 0, st>>>(DS, s, HUb, Ub, Cb + s * s + s, f);
      PF_LAUNCH_CHECK("corr_resid_kernel");
      FilterItem it;
      it.H = H;
      it.owner = this;
      it.prec = PF_F32;
      it.s = s;
      it.V = f;
      it.W = f + DS;
      it.colcoef = gam;
      it.K = Kr - 1;
      it.aux0 = f + 2 * DS;
      it.aux1 = f + 3 * DS;
      while ((int)g_refine.size() <= b) g_refine.emplace_back(new FilterGraph());
      it.graph = g_refine[b].get();
      pending.push_back(it);
      S.rep.filter_steps_f32 += Kr;
      S.rep.filter_steps_f64 += 1;
    }
    return PF_OK;
  }

  pf_status refine_post() {
    clk->mark(3);
    const int64_t DS = H->D * s;
    double* Ud = U.as<double>();
    double* HUd = HU.as<double>();
    double* Wd = HUd + (int64_t)Lb * DS;
    const bool corr = corr_form();
    if (refine_prec() == PF_DF64 && !corr && na > 0)   // W (pairs, over the active U blocks) to FP64
      PF_TRY(convert_df2d(reinterpret_cast<const float2*>(Ud + (int64_t)Lb * DS), Wd, na * DS, st));
    if (corr)   // W = P(theta) U + dW per active block, into the H U blocks as in the direct form
      for (int b = Lb; b < nb; ++b) {
        const double* pb = corr_small.as<double>() + (int64_t)b * (s * s + 2 * s) + s * s;
        const float* dW = reinterpret_cast<const float*>(aux64.as<double>() + (int64_t)(2 * b) * DS) + DS;
        corr_combine_kernel<<<(unsigned)ceil_div(DS, 256), 256, 0, st>>>(DS, s, Ud + (int64_t)b * DS, pb, dW,
                                                                         HUd + (int64_t)b * DS);
        PF_LAUNCH_CHECK("corr_combine_kernel");
      }
    if (Lb > 0) {   // the filtered blocks against the locked ones, two Gram-Schmidt passes
      DevBuf Cl;
      PF_TRY(Cl.alloc((size_t)Lb * s * na * s * 8, st));
      for (int pass = 0; pass < 2; ++pass) {
        PF_TRY((S.df ? gram_df : gram)(H->D, s, Ud, Lb, Wd, na, Cl.as<double>(), S.gscr.as<double>(), S.gscr_elems, st));
        for (int b = 0; b < na; ++b)
          PF_TRY((S.df ? tsgemm_df : tsgemm)(H->D, s, Ud, Lb, Cl.as<double>() + b * s, na * s, Wd + (int64_t)b * DS, 1, -1.0, 1.0, st));
      }
    }
    PF_TRY(orthonormalise_set(S, Wd, Ud + (int64_t)Lb * DS, na));
    PF_CUDA(cudaMemcpyAsync(Ud + (int64_t)Lb * DS, Wd, (size_t)na * DS * 8, cudaMemcpyDeviceToDevice, st));
    PF_TRY(rayleigh_ritz_H(S, Ud, HUd, nb, E, res));
    sel = nearest_sel(E, lam, nev);
    clk->mark(4);
    // the correction form's passes are FP32 steps (plus one FP64 step per block)
    (corr ? S.rep.ms_filter_f32 : S.rep.ms_filter_f64) += clk->ms(2, 3);
    S.rep.ms_refine += clk->ms(2, 4);
    if (passes < 8) {
      S.rep.refine_active[passes] = na;
      S.rep.refine_residual[passes] = max_res();
    }
    ++passes;
    const double cur = max_res();
    if (cur <= res_tol * hnorm || passes >= max_pass) return finish();
    // a stalled pass (gain under 2x) brings in the next reserve block, already in place in U.  A
    // lower bar (gain under 10x) let poorly filtered reserve vectors into the Rayleigh-Ritz of
    // low-degree, many-pair solves (XXZ L=14-16, nev=200, K=40-57), where a spurious Ritz pair
    // near the target then took a place in the returned set (residual 0.07-0.12 ||H||).
    if (cur > 0.5 * prev && nb < nb_total) ++nb;
    if (cur > 0.5 * prev && Kr < K && o.refine_K <= 0) {
      // the shorter default degree stalled (its wider lobe separates the set's edge too little
      // for this spectrum): the remaining passes use the Lanczos degree K
      Kr = K;
      coeffs_r.assign(Kr + 1, 0.0);
      PF_TRY(filter_coefficients_dev(lam_t, Kr, coeffs_r.data(), st));
      a0 = coeffs_r[0];
    }
    prev = cur;
    return issue_refine_filter();
  }

  pf_status finish() {
    phase = DONE;
    S.rep.refine_passes = passes;
    PF_CUDA(cudaEventRecord(t_end, st));
    PF_CUDA(cudaEventSynchronize(t_end));
    float tot = 0;
    cudaEventElapsedTime(&tot, t_begin, t_end);
    S.rep.ms_total = tot;
    S.rep.max_residual = max_res();
    S.rep.converged = 0;
    for (int j : sel) S.rep.converged += res[j] <= res_tol * hnorm;
    status = S.rep.converged == nev ? PF_OK : PF_ENOTCONV;
    S.rep.status = status;
    return PF_OK;
  }

  // evals/resid host [nev] (may be NULL), evecs device D x nev column-major (may be NULL).
  pf_status outputs(double* evals, double* evecs, double* resid, pf_report* rep) {
    if (phase != DONE || sel.size() != (size_t)nev) return status != PF_OK ? status : PF_ESTATE;
    for (int j = 0; j < nev; ++j) {
      if (evals) evals[j] = E[sel[j]];
      if (resid) resid[j] = res[sel[j]];
    }
    if (evecs) {
      DevBuf sd;
      PF_TRY(sd.alloc(nev * sizeof(int), st));
      PF_CUDA(cudaMemcpyAsync(sd.p, sel.data(), nev * sizeof(int), cudaMemcpyHostToDevice, st));
      gather_cols_kernel<<<(unsigned)ceil_div(H->D * nev, 256), 256, 0, st>>>(H->D, s, U.as<double>(), sd.as<int>(),
                                                                              nev, evecs);
      PF_LAUNCH_CHECK("gather_cols_kernel");
      PF_CUDA(cudaStreamSynchronize(st));
    }
    if (rep) *rep = S.rep;
    return status;
  }
};

// Device bytes a solve holds at its peak besides the Hamiltonian: the resident Lanczos
// state of solver_init, the Ritz set with H times it, and the FP32 path's refinement
// auxiliaries, plus the transient Rayleigh-Ritz matrices.  Mirrors the allocations above.
static size_t solve_state_bytes(int64_t D, int s, int nev, bool f32) {
  int nev_g = std::max(nev, (int)std::ceil(guard_factor((double)D) * nev));
  if (nev_g > D) nev_g = (int)D;
  const int Mmax = (int)std::min<int64_t>(expected_krylov_dim(nev_g, s, 1.5), D);
  int mb = std::max(2, Mmax / s);
  if ((int64_t)mb * s > D) mb = (int)(D / s);
  const int64_t Mcap = (int64_t)(mb + 1) * s;
  const int qb = (nev_g + s - 1) / s;
  const int qmax = std::max(qb * s + (f32 ? 2 * s : 0), nev_g);
  const int nbt = (qmax + s - 1) / s;
  const int64_t blk = D * s;
  size_t b = (size_t)(mb + 1) * blk * 8;                    // Krylov basis
  b += (size_t)Mcap * Mcap * 8;                             // H_L
  b += (size_t)blk * 8 * 2;                                 // W, tmp
  b += f32 ? (size_t)blk * 4 * 4 : (size_t)blk * 8 * 2;     // aux pair (+ V32, W32)
  b += std::max(gram_scratch_elems(D, s, mb + 1, 1), gram_scratch_elems(D, s, nbt, nbt)) * 8;
  b += eig_workspace_bytes((int)Mcap, std::max(qmax, 2)) + (size_t)Mcap * std::max(qmax, 2) * 8 * 2;
  b += (size_t)nbt * blk * 8 * 2;                           // U, H U
  if (f32) b += (size_t)2 * nbt * blk * 8;                  // refinement auxiliaries
  b += (size_t)qmax * qmax * 8 * 5 + eig_workspace_bytes(qmax, qmax);   // Rayleigh-Ritz
  return b + ((size_t)16 << 20);
}

// Runs the pending filter applications of a set of tasks and then each task's follow-up.
// Items with equal (precision, block width) form one group: a group of one item runs the
// plain K-step recurrence, larger groups run one sweep (one launch per Clenshaw step over
// all their rows).  A task whose follow-up fails is marked done with that status; the others
// continue.
struct Executor {
  DevBuf table;
  std::vector<unsigned char> table_host;
  SweepGraph graph;
  cudaStream_t st = 0;
  int force_csize = -1;   // -1: the autotuner decides per group of one shape; >= 0: that form for every group

  pf_status run_group(const std::vector<FilterItem>& items, int csize) {
    if (items.empty()) return PF_OK;
    if (items.size() == 1 && csize == 0) {
      const FilterItem& it = items[0];
      return filter_apply_raw(it.H, it.prec, it.s, it.V, it.W, it.coeffs_host, it.colcoef, it.K, it.aux0, it.aux1, st);
    }
    const size_t need = filter_sweep_table_bytes((int)items.size());
    if (table.bytes < need) PF_TRY(table.alloc(need * 2, st));
    if (table_host.size() < need) table_host.resize(need * 2);
    // table_host is pageable: the copy inside has consumed it when the call returns.
    return filter_sweep(items, table.p, table.bytes, table_host.data(), st, csize, csize == 0 ? &graph : nullptr);
  }

  pf_status run_round(std::vector<Task*>& tasks) {
    std::vector<std::pair<std::pair<int, int>, std::vector<FilterItem>>> groups;
    for (Task* t : tasks) {
      if (t->phase == Task::DONE) continue;
      for (const FilterItem& it : t->pending) {
        if (it.colcoef) {   // per-column coefficients: the plain recurrence, alone
          PF_TRY(run_group(std::vector<FilterItem>(1, it), 0));
          continue;
        }
        const auto key = std::make_pair(it.prec, it.s);
        auto g = std::find_if(groups.begin(), groups.end(), [&](const auto& x) { return x.first == key; });
        if (g == groups.end()) {
          groups.push_back({key, {}});
          g = groups.end() - 1;
        }
        g->second.push_back(it);
      }
    }
    for (auto& g : groups) {
      // items of one shape (same D and nnz) form a subgroup; the autotuner picks its form
      std::vector<std::pair<std::pair<int64_t, int64_t>, std::vector<FilterItem>>> shapes;
      for (const FilterItem& it : g.second) {
        const auto key = std::make_pair(it.H->D, it.H->nnz);
        auto p = std::find_if(shapes.begin(), shapes.end(), [&](const auto& x) { return x.first == key; });
        if (p == shapes.end()) {
          shapes.push_back({key, {}});
          p = shapes.end() - 1;
        }
        p->second.push_back(it);
      }
      for (auto& p : shapes) {
        const auto& items = p.second;
        int c = force_csize;
        if (c < 0) {
          TuneResult tr;
          PF_TRY(tune_item(items[0], st, &tr));
          c = choose_form(tr, (int)items.size(), nullptr);
        }
        bool one_owner = true;
        for (const FilterItem& it : items) one_owner = one_owner && it.owner == items[0].owner;
        if (c == 0 && (items.size() == 1 || one_owner)) {
          // one item, or the blocks of one solve (refinement): the plain recurrence per item
          // keeps the step kernel's specialised form; sweeps pay off across solves
          for (const FilterItem& it : items) PF_TRY(run_group(std::vector<FilterItem>(1, it), 0));
        } else {
          PF_TRY(run_group(items, c));
        }
      }
    }
    for (Task* t : tasks) {
      if (t->phase == Task::DONE || t->pending.empty()) continue;
      const pf_status s = t->after_filter();
      if (s != PF_OK) {
        t->status = s;
        t->phase = Task::DONE;
        t->pending.clear();
      }
    }
    return PF_OK;
  }

  pf_status run(std::vector<Task*>& tasks) {
    for (;;) {
      bool any = false;
      for (Task* t : tasks) any = any || (t->phase != Task::DONE && !t->pending.empty());
      if (!any) return PF_OK;
      PF_TRY(run_round(tasks));
    }
  }
};

// ------------------------------------------------------------------ asynchronous executor
// Drives many solves from one host thread without rounds: each solve runs on its own stream
// (from a process-wide pool), a finished filter application is noticed by polling its event,
// and the solve's follow-up work is issued at once, so solves in different phases overlap on
// the device (an FP64 refinement pass, bound by the FP64 pipe, beside another solve's FP32
// Lanczos steps, bound by memory).  Filter applications are queued as captured graphs (one
// call per application).  Items of one shape that are ready together still share a sweep or
// a persistent launch (as chosen by the autotuner), issued on a group stream that waits for
// the solves' streams and that they wait for in turn.
//
// Start gate: a solve whose FP32 step working set exceeds a third of L2 starts its Lanczos
// phase only while no other such solve is in its Lanczos phase.  Two of them would evict each
// other's working set from L2 with no gain in throughput; staggered, the next one's Lanczos
// phase overlaps the previous one's refinement.
namespace {
std::mutex g_pool_mu;
struct StreamPool {
  std::vector<cudaStream_t> s;
  cudaStream_t group = nullptr;
};
std::map<int, StreamPool> g_pools;
constexpr int kPoolStreams = 16;
}  // namespace

// Streams live for the process: memory that a caching allocator keeps per stream stays usable
// by the next batch or server.
static pf_status pool_streams(StreamPool** out) {
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_pool_mu);
  StreamPool& p = g_pools[dev];
  if (p.s.empty()) {
    for (int i = 0; i < kPoolStreams; ++i) {
      cudaStream_t x;
      PF_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
      p.s.push_back(x);
    }
    PF_CUDA(cudaStreamCreateWithFlags(&p.group, cudaStreamNonBlocking));
  }
  *out = &p;
  return PF_OK;
}

// Pinned host staging for sweep tables: a slot is reused once the copy that read it is done.
struct PinnedRing {
  struct Slot {
    void* p = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
  };
  std::vector<Slot> slots;
  ~PinnedRing() {
    for (auto& x : slots) {
      if (x.ev) cudaEventSynchronize(x.ev), cudaEventDestroy(x.ev);
      if (x.p) cudaFreeHost(x.p);
    }
  }
  pf_status get(size_t bytes, Slot** out) {
    for (auto& x : slots) {
      if (x.bytes >= bytes && cudaEventQuery(x.ev) == cudaSuccess) {
        *out = &x;
        return PF_OK;
      }
    }
    cudaGetLastError();
    slots.emplace_back();
    Slot& x = slots.back();
    PF_CUDA(cudaMallocHost(&x.p, std::max<size_t>(bytes, 4096)));
    x.bytes = std::max<size_t>(bytes, 4096);
    PF_CUDA(cudaEventCreateWithFlags(&x.ev, cudaEventDisableTiming));
    *out = &x;
    return PF_OK;
  }
};

// FP32 step working set (three D x s blocks and the FP32 CSR) above a third of L2.
static bool l2_heavy(const Ham* H, const pf_solve_opts& o) {
  if (o.precision != PF_F32 || !H) return false;
  const int s = o.block > 0 ? o.block : 32;
  const double ws = (double)H->D * s * 4 * 3 + (double)H->nnz * 8;
  return ws > 42e6;
}

struct AsyncExecutor {
  struct Live {
    Task* t = nullptr;
    std::function<pf_status(Task*, cudaStream_t)> start;   // init, deferred by the start gate
    bool heavy = false, started = false, inflight = false;
    cudaEvent_t done = nullptr, ready = nullptr;
    cudaStream_t st = nullptr;
  };
  std::vector<Live> live;
  StreamPool* pool = nullptr;
  DevBuf table;
  PinnedRing ring;
  SweepGraph sgraph;
  int next_stream = 0;

  ~AsyncExecutor() {
    for (auto& l : live) {
      if (l.done) cudaEventDestroy(l.done);
      if (l.ready) cudaEventDestroy(l.ready);
    }
  }
  pf_status setup() { return pool_streams(&pool); }

  // Registers a solve; `start` initialises it on the stream it is given.
  pf_status add(Task* t, bool heavy, std::function<pf_status(Task*, cudaStream_t)> start) {
    Live l;
    l.t = t;
    l.heavy = heavy;
    l.start = std::move(start);
    PF_CUDA(cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming));
    PF_CUDA(cudaEventCreateWithFlags(&l.ready, cudaEventDisableTiming));
    l.st = pool->s[next_stream++ % kPoolStreams];
    live.push_back(l);
    return PF_OK;
  }

  void fail(Live& l, pf_status s) {
    l.t->status = s;
    l.t->phase = Task::DONE;
    l.t->pending.clear();
    l.inflight = false;
    l.started = true;
  }

  bool finished(const Live& l) const { return l.started && l.t->phase == Task::DONE; }
  bool is_finished(const Task* t) const {
    for (const auto& l : live)
      if (l.t == t) return finished(l);
    return true;
  }
  void remove(const Task* t) {
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i].t == t) {
        if (live[i].done) cudaEventDestroy(live[i].done);
        if (live[i].ready) cudaEventDestroy(live[i].ready);
        live.erase(live.begin() + i);
        return;
      }
  }
  bool all_done() const {
    for (const auto& l : live)
      if (!finished(l)) return false;
    return true;
  }

  // Starts solves the gate admits, in registration order.
  void start_ready() {
    int heavy_lanczos = 0;
    for (const auto& l : live)
      if (l.started && l.heavy && l.t->phase == Task::LANCZOS) ++heavy_lanczos;
    for (auto& l : live) {
      if (l.started) continue;
      if (l.heavy && heavy_lanczos > 0) continue;
      l.t->captured = true;
      const pf_status s = l.start(l.t, l.st);
      l.started = true;
      if (s != PF_OK) {
        fail(l, s);
        continue;
      }
      if (l.heavy && l.t->phase == Task::LANCZOS) ++heavy_lanczos;
    }
  }

  // Issues the pending filter applications of every started, idle solve.
  pf_status launch_ready() {
    std::vector<Live*> idle;
    for (auto& l : live)
      if (l.started && !l.inflight && l.t->phase != Task::DONE && !l.t->pending.empty()) idle.push_back(&l);
    if (idle.empty()) return PF_OK;
    // shape groups across solves: (prec, s, D, nnz)
    struct Grp {
      int prec, s;
      int64_t D, nnz;
      std::vector<std::pair<FilterItem, Live*>> items;
    };
    // Overlap: while one solve runs its FP32 Lanczos phase and another its refinement, their
    // large steps are capped at 3 (FP32) and 4 (FP64) or 2 (pair-float) CTAs per SM, which fit
    // together in one SM's registers (3 x 256 x 40 + 4 x 256 x 32, or + 2 x 256 x 54, of 65536)
    // and thread slots, so both kinds of step share every SM instead of queueing for slots.
    bool lanczos32 = false, refine64 = false;
    for (const auto& l : live) {
      if (!l.started || l.t->phase == Task::DONE) continue;
      lanczos32 = lanczos32 || (l.t->phase == Task::LANCZOS && l.t->f32 && l.heavy);
      refine64 = refine64 || (l.t->phase == Task::REFINE && l.heavy);
    }
    const bool overlap = lanczos32 && refine64;
    for (Live* l : idle)
      for (FilterItem& it : l->t->pending) {
        const double blk = (double)it.H->D * it.s * prec_bytes(it.prec);
        it.cta_cap = (overlap && blk >= 16e6) ? (it.prec == PF_F64 ? 4 : it.prec == PF_DF64 ? 2 : 3) : 0;
      }
    std::vector<Grp> grps;
    for (Live* l : idle)
      for (const FilterItem& it : l->t->pending) {
        if (it.colcoef) {   // per-column coefficients: its captured recurrence, alone
          PF_TRY(filter_graph_launch(*it.graph, it, l->st));
          continue;
        }
        auto g = std::find_if(grps.begin(), grps.end(), [&](const Grp& x) {
          return x.prec == it.prec && x.s == it.s && x.D == it.H->D && x.nnz == it.H->nnz;
        });
        if (g == grps.end()) {
          grps.push_back(Grp{it.prec, it.s, it.H->D, it.H->nnz, {}});
          g = grps.end() - 1;
        }
        g->items.push_back({it, l});
      }
    for (auto& g : grps) {
      TuneResult tr;
      PF_TRY(tune_item(g.items[0].first, g.items[0].second->st, &tr));
      const int n = (int)g.items.size();
      const int c = choose_form(tr, n, nullptr);
      bool one_owner = true;
      for (auto& x : g.items) one_owner = one_owner && x.second == g.items[0].second;
      if (c == 0 && (n == 1 || one_owner)) {
        for (auto& x : g.items) PF_TRY(filter_graph_launch(*x.first.graph, x.first, x.second->st));
        continue;
      }
      // one launch (sweep or persistent) for the group on the group stream
      std::vector<Live*> owners;
      for (auto& x : g.items)
        if (std::find(owners.begin(), owners.end(), x.second) == owners.end()) owners.push_back(x.second);
      for (Live* l : owners) {
        PF_CUDA(cudaEventRecord(l->ready, l->st));
        PF_CUDA(cudaStreamWaitEvent(pool->group, l->ready, 0));
      }
      std::vector<FilterItem> items;
      for (auto& x : g.items) items.push_back(x.first);
      const size_t need = filter_sweep_table_bytes(n);
      if (table.bytes < need) {
        PF_CUDA(cudaStreamSynchronize(pool->group));
        PF_TRY(table.alloc(need * 4, pool->group));
      }
      PinnedRing::Slot* slot = nullptr;
      PF_TRY(ring.get(need, &slot));
      PF_TRY(filter_sweep(items, table.p, table.bytes, slot->p, pool->group, c, c == 0 ? &sgraph : nullptr));
      PF_CUDA(cudaEventRecord(slot->ev, pool->group));
      for (Live* l : owners) PF_CUDA(cudaStreamWaitEvent(l->st, slot->ev, 0));
    }
    for (Live* l : idle) {
      PF_CUDA(cudaEventRecord(l->done, l->st));
      l->inflight = true;
    }
    return PF_OK;
  }

  // Runs the follow-up of every solve whose filter application has finished.  With `wait`,
  // sleeps briefly when nothing has finished yet.
  pf_status poll(bool wait, int* completed) {
    int done = 0;
    for (auto& l : live) {
      if (!l.inflight) continue;
      const cudaError_t q = cudaEventQuery(l.done);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        set_cuda_error(q, "cudaEventQuery");
        return PF_ECUDA;
      }
      l.inflight = false;
      ++done;
      const pf_status s = l.t->after_filter();
      if (s != PF_OK) fail(l, s);
    }
    cudaGetLastError();
    if (!done && wait) std::this_thread::sleep_for(std::chrono::microseconds(50));
    if (completed) *completed = done;
    return PF_OK;
  }

  pf_status run() {
    while (!all_done()) {
      start_ready();
      PF_TRY(launch_ready());
      PF_TRY(poll(true, nullptr));
    }
    return PF_OK;
  }
};

static pf_status polfed_solve_impl(Ham* H, double target_eps, int nev, int K, const pf_solve_opts* o_in,
                                   double* evals, double* evecs, double* resid, pf_report* rep, cudaStream_t st) {
  if (!H || !evals || !resid) return PF_EINVAL;
  Task t;
  PF_TRY(t.init(H, target_eps, nev, K, o_in, st));
  Executor ex;
  ex.st = st;
  std::vector<Task*> v{&t};
  PF_TRY(ex.run(v));
  if (t.phase != Task::DONE || t.sel.empty()) return t.status != PF_OK ? t.status : PF_ENOTCONV;
  return t.outputs(evals, evecs, resid, rep);
}

// ------------------------------------------------------------------ serving
// Continuous batching.  Requests queue on submit.  Each step admits queued requests in
// arrival order while the sum of the admitted footprints stays within the budget (the
// first request is admitted into an empty server whatever its size), builds their basis,
// Hamiltonian, bounds and K, runs one executor round over all resident solves (their
// filter applications share sweeps) and retires the finished ones, releasing their memory.
struct Request {
  int64_t id = 0;
  pf_model m;
  std::vector<double> h, mu, A, un, E;
  std::vector<int32_t> nj;
  double eps = 0.5;
  int nev = 1;
  int state = 0;   // 0 queued, 1 active, 2 finished
  pf_status status = PF_OK;
  size_t foot = 0;
  pf_basis* basis = nullptr;
  pf_ham* ham = nullptr;
  Task* task = nullptr;
  std::vector<double> evals, resid;
  pf_report rep;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int64_t model_dim(const pf_model& m) {
  auto C = [](int n, int k) -> double {
    if (k < 0 || k > n) return 0;
    double r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return std::floor(r + 0.5);
  };
  if (m.kind == PF_MODEL_XXZ) return (int64_t)C(m.L, m.N);
  if (m.kind == PF_MODEL_HUBBARD) return (int64_t)(C(m.L, m.N_up) * C(m.L, m.N_dn));
  if (m.kind == PF_MODEL_QSUN) return (int64_t)1 << (m.N + m.L);
  if (m.kind == PF_MODEL_QREM) return (int64_t)1 << m.L;
  if (m.kind == PF_MODEL_QSUN_U1) return (int64_t)C(m.N + m.L, m.N_up);
  return 0;
}

// Stored entries per row, an upper bound: the diagonal plus one per bond (XXZ), two per bond
// (Hubbard), the dot block plus one per outer spin (quantum sun).
static int64_t model_nnz_bound(const pf_model& m, int64_t D) {
  if (m.kind == PF_MODEL_XXZ) return D * (1 + m.L * (1 + (m.J2 != 0.0) + (m.J3 != 0.0)));
  if (m.kind == PF_MODEL_HUBBARD) return D * (1 + 2 * m.L);
  if (m.kind == PF_MODEL_QREM) return D * (1 + m.L);
  return D * (((int64_t)1 << m.N) + m.L);
}

// row_ptr, col + the four value arrays (H, H~ in FP64, FP32, pairs), the basis states, and
// the structured mapping's diagonal in three forms
static size_t ham_bytes(int64_t D, int64_t nnz) { return (size_t)(D + 1) * 8 + (size_t)nnz * 32 + (size_t)D * 24; }

struct Server {
  pf_server_config cfg;
  cudaStream_t st = 0;
  int64_t next_id = 1;
  std::vector<Request*> queue, active, finished;
  size_t in_use = 0;
  AsyncExecutor ex;
  bool ready = false;

  ~Server() {
    for (auto* v : {&queue, &active, &finished})
      for (Request* r : *v) {
        release(r);
        delete r;
      }
  }
  void release(Request* r) {
    if (r->task) {
      cudaStream_t s = r->task->st;
      ex.remove(r->task);
      delete r->task;
      r->task = nullptr;
      if (s) cudaStreamSynchronize(s);
    }
    if (r->ham) pf_free_ham(r->ham);
    if (r->basis) pf_free_basis(r->basis);
    r->ham = nullptr;
    r->basis = nullptr;
  }
  pf_solve_opts opts() const {
    pf_solve_opts o;
    pf_default_opts(&o);
    o.block = cfg.block;
    o.precision = cfg.precision;
    if (cfg.res_tol > 0) o.res_tol = cfg.res_tol;
    if (cfg.seed) o.seed = cfg.seed;
    o.refine_precision = cfg.refine_precision;
    o.refine_form = cfg.refine_form;
    return o;
  }
  // Admission work, on the stream the executor gives the solve: basis, Hamiltonian, bounds,
  // K, then the solve's initialisation.
  pf_status start(Request* r, Task* t, cudaStream_t s) {
    pf_params p;
    memset(&p, 0, sizeof(p));
    p.h = r->h.empty() ? nullptr : r->h.data();
    p.mu = r->mu.empty() ? nullptr : r->mu.data();
    p.A = r->A.empty() ? nullptr : r->A.data();
    p.u_noise = r->un.empty() ? nullptr : r->un.data();
    p.n_of_j = r->nj.empty() ? nullptr : r->nj.data();
    p.E = r->E.empty() ? nullptr : r->E.data();
    r->t_admit = now_ms();
    PF_TRY(pf_build_basis(&r->m, &r->basis, s));
    PF_TRY(pf_build_hamiltonian(r->basis, &r->m, &p, &r->ham, s));
    double emin, emax;
    PF_TRY(pf_spectral_bounds(r->ham, cfg.bounds_tol, &emin, &emax, nullptr, nullptr, s));
    int32_t K = 0;
    PF_TRY(pf_choose_K(r->ham, r->eps, r->nev, &K, s));
    const pf_solve_opts o = opts();
    return t->init(reinterpret_cast<Ham*>(r->ham), r->eps, r->nev, K, &o, s);
  }
  void retire(Request* r, pf_status s) {
    r->status = s;
    r->state = 2;
    r->t_done = now_ms();
    in_use -= r->foot;
    release(r);
    finished.push_back(r);
  }
  pf_status step(int32_t* nq, int32_t* na, int32_t* nf) {
    if (!ready) {
      PF_TRY(ex.setup());
      ready = true;
    }
    while (!queue.empty() && (int)active.size() < cfg.max_active) {
      Request* r = queue.front();
      if (!active.empty() && in_use + r->foot > (size_t)cfg.mem_budget_bytes) break;
      queue.erase(queue.begin());
      r->state = 1;
      in_use += r->foot;
      r->task = new Task();
      const pf_solve_opts o = opts();
      const int64_t D = model_dim(r->m);
      Ham probe;
      probe.D = D;
      probe.nnz = model_nnz_bound(r->m, D);
      PF_TRY(ex.add(r->task, l2_heavy(&probe, o), [this, r](Task* t, cudaStream_t s) { return start(r, t, s); }));
      active.push_back(r);
    }
    ex.start_ready();
    PF_TRY(ex.launch_ready());
    PF_TRY(ex.poll(true, nullptr));
    for (size_t i = 0; i < active.size();) {
      Request* r = active[i];
      if (ex.is_finished(r->task)) {
        r->evals.assign(r->nev, 0.0);
        r->resid.assign(r->nev, 0.0);
        memset(&r->rep, 0, sizeof(r->rep));
        const pf_status s = r->task->outputs(r->evals.data(), nullptr, r->resid.data(), &r->rep);
        active.erase(active.begin() + i);
        retire(r, s);
      } else {
        ++i;
      }
    }
    if (nq) *nq = (int32_t)queue.size();
    if (na) *na = (int32_t)active.size();
    if (nf) *nf = (int32_t)finished.size();
    return PF_OK;
  }
};

static pf_status copy_request(const pf_model* m, const pf_params* p, Request* r) {
  r->m = *m;
  const int L = m->L;
  if (L < 1 || L > 32) return PF_EINVAL;
  if (m->kind == PF_MODEL_XXZ) {
    if (!p->h) return PF_EINVAL;
    r->h.assign(p->h, p->h + L);
  } else if (m->kind == PF_MODEL_HUBBARD) {
    if (!p->mu) return PF_EINVAL;
    r->mu.assign(p->mu, p->mu + L);
  } else if (m->kind == PF_MODEL_QSUN || m->kind == PF_MODEL_QSUN_U1) {
    if (!p->h || !p->A || !p->u_noise || !p->n_of_j || m->N < 1 || m->N > 10) return PF_EINVAL;
    const int nd = 1 << m->N;
    r->h.assign(p->h, p->h + L);
    r->A.assign(p->A, p->A + (size_t)nd * nd);
    r->un.assign(p->u_noise, p->u_noise + L);
    r->nj.assign(p->n_of_j, p->n_of_j + L);
  } else if (m->kind == PF_MODEL_QREM) {
    if (!p->E || L > 30) return PF_EINVAL;
    r->E.assign(p->E, p->E + ((size_t)1 << L));
  } else {
    return PF_EINVAL;
  }
  return PF_OK;
}

}  // namespace pf

using namespace pf;

struct pf_server : pf::Server {};

extern "C" {

void pf_default_opts(pf_solve_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->block = 32;
  o->precision = PF_F64;
  o->eta = 1.5;
  o->tol = 1e-10;
  o->tol_f32 = 1e-7;
  o->res_tol = 1e-9;
  o->seed = 2024;
  o->refine_precision = PF_F64;
}

pf_status pf_spectral_bounds(pf_ham* hh, double tol, double* emin, double* emax, double* rmin, double* rmax,
                             pf_stream_t stream) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H || !emin || !emax) return PF_EINVAL;
  PF_TRY(spectral_bounds_impl(H, tol, (cudaStream_t)stream));
  *emin = H->emin;
  *emax = H->emax;
  if (rmin) *rmin = H->rmin;
  if (rmax) *rmax = H->rmax;
  return PF_OK;
}

pf_status pf_filter_coefficients(double lam_t, int32_t K, double* coeffs, pf_stream_t stream) {
  if (K < 1 || !coeffs || !(lam_t >= -1.0 && lam_t <= 1.0)) return PF_EINVAL;
  return filter_coefficients_dev(lam_t, K, coeffs, (cudaStream_t)stream);
}

pf_status pf_choose_K(pf_ham* hh, double target_eps, int32_t nev, int32_t* K, pf_stream_t stream) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H || !K || nev < 1) return PF_EINVAL;
  if (!H->has_bounds || !H->has_rescale) return PF_ESTATE;
  if (!(target_eps >= 0.0 && target_eps <= 1.0)) return PF_EINVAL;
  double mu = 0, G = 0;
  PF_TRY(ham_moments(H, &mu, &G, (cudaStream_t)stream));
  const double lam = H->emin + target_eps * (H->emax - H->emin);
  const double lt = (lam - H->Ec) / H->dE;
  const int nev_g = (int)std::ceil(guard_factor((double)H->D) * nev);
  const double rho = (double)H->D / (std::sqrt(2.0 * M_PI) * G) * std::exp(-(lt - mu) * (lt - mu) / (2.0 * G * G));
  const double delta = nev_g / (2.0 * rho);
  const double k = 2.655 * std::sqrt(std::max(1.0 - lt * lt, 0.0)) / delta;
  *K = std::max(1, (int)std::ceil(k));
  return PF_OK;
}

pf_status pf_polfed_solve(pf_ham* hh, double target_eps, int32_t nev, int32_t K, const pf_solve_opts* o,
                          double* evals, double* evecs, double* resid, pf_report* rep, pf_stream_t stream) {
  return polfed_solve_impl(reinterpret_cast<Ham*>(hh), target_eps, nev, K, o, evals, evecs, resid, rep,
                           (cudaStream_t)stream);
}

// z = x + i y from column `col` of the real embedding's eigenvectors (2 Dc rows, column-major),
// written as (re, im) pairs into column k of Z (Dc complex entries per column).
__global__ void complex_column_kernel(int64_t Dc, const double* V2, int col, double* Z, int k) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= Dc) return;
  const double* v = V2 + (int64_t)col * 2 * Dc;
  Z[((int64_t)k * Dc + r) * 2] = v[r];
  Z[((int64_t)k * Dc + r) * 2 + 1] = v[Dc + r];
}

pf_status pf_polfed_solve_complex(pf_ham* hh, double target_eps, int32_t nev, int32_t K, const pf_solve_opts* o,
                                  double* evals, double* evecs, double* resid, pf_report* rep, pf_stream_t stream) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H || !evals || !resid) return PF_EINVAL;
  if (H->Dc <= 0 || nev < 1 || 2 * (int64_t)nev > H->D) return PF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // every eigenvalue of H appears twice in the embedding: solve for 2 nev
  const int n2 = 2 * nev;
  std::vector<double> e2(n2), r2(n2);
  DevBuf v2;
  if (evecs) PF_TRY(v2.alloc((size_t)H->D * n2 * sizeof(double), st));
  pf_report rp;
  const pf_status s = polfed_solve_impl(H, target_eps, n2, K, o, e2.data(), evecs ? v2.as<double>() : nullptr,
                                        r2.data(), &rp, st);
  if (s != PF_OK && s != PF_ENOTCONV) return s;
  if (rep) *rep = rp;
  // the 2 nev values come ascending as pairs of copies; a pair whose copies disagree by more than
  // the residual tolerance, or two pairs that coincide (a degenerate eigenvalue of H), cannot be
  // matched to distinct eigenvectors of H
  const double tol = (o && o->res_tol > 0 ? o->res_tol : 1e-9) * rp.hnorm;
  for (int k = 0; k < nev; ++k) {
    if (std::fabs(e2[2 * k + 1] - e2[2 * k]) > tol) return PF_EBREAKDOWN;
    if (k + 1 < nev && e2[2 * k + 2] - e2[2 * k + 1] <= tol) return PF_EBREAKDOWN;
  }
  for (int k = 0; k < nev; ++k) {
    const int c = r2[2 * k + 1] < r2[2 * k] ? 2 * k + 1 : 2 * k;   // the copy with the smaller residual
    evals[k] = e2[c];
    resid[k] = r2[c];
    if (evecs) {
      complex_column_kernel<<<(unsigned)ceil_div(H->Dc, 256), 256, 0, st>>>(H->Dc, v2.as<double>(), c, evecs, k);
      PF_LAUNCH_CHECK("complex_column_kernel");
    }
  }
  if (evecs) PF_CUDA(cudaStreamSynchronize(st));
  return s;
}

pf_status pf_polfed_solve_batch(pf_solve_item* items, int32_t n, pf_stream_t stream) {
  if (n < 0 || (n > 0 && !items)) return PF_EINVAL;
  if (n == 0) return PF_OK;
  // the solves run on the library's stream pool; the caller's stream is drained first so
  // that work the caller queued before (bounds, buffers) is complete
  PF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  AsyncExecutor ex;
  PF_TRY(ex.setup());
  std::vector<std::unique_ptr<Task>> tasks;
  std::vector<int> slot;
  for (int i = 0; i < n; ++i) {
    pf_solve_item& it = items[i];
    it.status = PF_OK;
    if (!it.H || !it.evals || !it.resid) {
      it.status = PF_EINVAL;
      continue;
    }
    pf_solve_opts o;
    pf_default_opts(&o);
    if (it.opts) o = *it.opts;
    Ham* H = reinterpret_cast<Ham*>(it.H);
    const double eps = it.target_eps;
    const int nev = it.nev, K = it.K;
    tasks.emplace_back(new Task());
    slot.push_back(i);
    PF_TRY(ex.add(tasks.back().get(), l2_heavy(H, o), [H, eps, nev, K, o](Task* t, cudaStream_t st) {
      return t->init(H, eps, nev, K, &o, st);
    }));
  }
  pf_status rs = ex.run();
  pf_status first_bad = PF_OK;
  for (size_t j = 0; j < tasks.size(); ++j) {
    pf_solve_item& it = items[slot[j]];
    Task* t = tasks[j].get();
    if (rs != PF_OK) it.status = rs;   // a shared launch failed: every problem reports it
    else
      it.status = (t->phase == Task::DONE && !t->sel.empty()) ? t->outputs(it.evals, it.evecs, it.resid, it.rep)
                                                              : (t->status != PF_OK ? t->status : PF_ENOTCONV);
  }
  for (auto& t : tasks) {   // release on the solves' own streams before the executor goes
    cudaStream_t st = t->st;
    t.reset();
    if (st) cudaStreamSynchronize(st);
  }
  for (int i = 0; i < n; ++i)
    if (items[i].status != PF_OK && first_bad == PF_OK) first_bad = (pf_status)items[i].status;
  return rs != PF_OK ? rs : first_bad;
}

pf_status pf_solve_footprint(int64_t D, int64_t nnz, int32_t nev, int32_t block, int32_t precision,
                             int64_t* bytes) {
  if (D < 1 || nnz < 0 || nev < 1 || nev > D || !bytes) return PF_EINVAL;
  const int s = block > 0 ? block : 32;
  if (!(s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32 || s == 64)) return PF_EINVAL;
  if (precision != PF_F64 && precision != PF_F32) return PF_EINVAL;
  *bytes = (int64_t)(ham_bytes(D, nnz) + solve_state_bytes(D, s, nev, precision == PF_F32));
  return PF_OK;
}

pf_status pf_server_create(const pf_server_config* cfg, pf_stream_t stream, pf_server** out) {
  if (!out) return PF_EINVAL;
  *out = nullptr;
  pf_server_config c;
  memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  if (c.block == 0) c.block = 32;
  if (!(c.block < 0 || c.block == 1 || c.block == 2 || c.block == 4 || c.block == 8 || c.block == 16 ||
        c.block == 32 || c.block == 64))
    return PF_EINVAL;
  if (c.precision != PF_F64 && c.precision != PF_F32) return PF_EINVAL;
  if (c.refine_precision != PF_F64 && c.refine_precision != PF_DF64) return PF_EINVAL;
  if (c.refine_form != 0 && c.refine_form != PF_REFINE_DIRECT && c.refine_form != PF_REFINE_CORRECTION) return PF_EINVAL;
  if (c.max_active <= 0) c.max_active = 64;
  if (c.mem_budget_bytes < 0) return PF_EINVAL;
  if (c.mem_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    PF_CUDA(cudaMemGetInfo(&fr, &tot));
    c.mem_budget_bytes = (int64_t)(0.8 * (double)fr);
  }
  pf_server* sv = new pf_server();
  sv->cfg = c;
  sv->st = (cudaStream_t)stream;
  *out = sv;
  return PF_OK;
}

pf_status pf_server_submit(pf_server* sv, const pf_model* m, const pf_params* p, double target_eps, int32_t nev,
                           int64_t* id) {
  if (!sv || !m || !p || !id) return PF_EINVAL;
  if (!(target_eps >= 0.0 && target_eps <= 1.0) || nev < 1) return PF_EINVAL;
  if (m->kind == PF_MODEL_XXZ && m->phi != 0.0) return PF_EINVAL;   // complex models: pf_polfed_solve_complex
  std::unique_ptr<Request> r(new Request());
  PF_TRY(copy_request(m, p, r.get()));
  const int64_t D = model_dim(*m);
  if (D < 1 || nev > D) return PF_EINVAL;
  r->eps = target_eps;
  r->nev = nev;
  const int sb = sv->cfg.block > 0 ? sv->cfg.block : 32;   // autotuned widths are estimated at 32
  r->foot = ham_bytes(D, model_nnz_bound(*m, D)) + solve_state_bytes(D, sb, nev, sv->cfg.precision == PF_F32);
  r->id = sv->next_id++;
  r->t_submit = now_ms();
  *id = r->id;
  sv->queue.push_back(r.release());
  return PF_OK;
}

pf_status pf_server_step(pf_server* sv, int32_t* queued, int32_t* active, int32_t* finished) {
  if (!sv) return PF_EINVAL;
  return sv->step(queued, active, finished);
}

pf_status pf_server_take(pf_server* sv, int64_t id, double* evals, double* resid, pf_report* rep,
                         pf_request_info* info) {
  if (!sv) return PF_EINVAL;
  for (size_t i = 0; i < sv->finished.size(); ++i) {
    Request* r = sv->finished[i];
    if (r->id != id) continue;
    if (evals && !r->evals.empty()) memcpy(evals, r->evals.data(), r->nev * sizeof(double));
    if (resid && !r->resid.empty()) memcpy(resid, r->resid.data(), r->nev * sizeof(double));
    if (rep) *rep = r->rep;
    if (info) {
      info->id = r->id;
      info->status = r->status;
      info->nev = r->nev;
      info->footprint_bytes = (int64_t)r->foot;
      info->queue_ms = r->t_admit - r->t_submit;
      info->latency_ms = r->t_done - r->t_submit;
    }
    sv->finished.erase(sv->finished.begin() + i);
    delete r;
    return PF_OK;
  }
  for (auto* v : {&sv->queue, &sv->active})
    for (Request* r : *v)
      if (r->id == id) return PF_ESTATE;
  return PF_EINVAL;
}

pf_status pf_server_memory(const pf_server* sv, int64_t* in_use, int64_t* budget) {
  if (!sv) return PF_EINVAL;
  if (in_use) *in_use = (int64_t)sv->in_use;
  if (budget) *budget = sv->cfg.mem_budget_bytes;
  return PF_OK;
}

void pf_server_destroy(pf_server* sv) { delete sv; }

pf_status pf_autotune_block(pf_ham* hh, int32_t precision, int32_t nev, int32_t* block, double* step_us,
                            double* cost, pf_stream_t stream) {
  Ham* H = reinterpret_cast<Ham*>(hh);
  if (!H || !block || nev < 1) return PF_EINVAL;
  if (precision != PF_F64 && precision != PF_F32) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  int s = 0;
  if (cost)
    for (int c = 0; c < 4; ++c) cost[c] = 0.0;
  PF_TRY(autotune_block(H, precision, nev, (cudaStream_t)stream, &s, step_us, cost));
  *block = s;
  return PF_OK;
}

pf_status pf_start_block(int64_t D, int32_t s, uint64_t seed, double* out, pf_stream_t stream) {
  if (D < 1 || s < 1 || !out) return PF_EINVAL;
  return start_block_raw(D, s, seed, out, (cudaStream_t)stream);
}

}  // extern "C"
