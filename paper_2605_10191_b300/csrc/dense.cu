// Tall-skinny FP64 kernels of the block-Lanczos loop (a6, a7, a9) and small dense
// helpers.  Blocked storage: a set of nb blocks, each D x s row-major, block b at
// X + b*D*s (the layout of the Krylov basis V_1..V_m and of Ritz-vector sets).
//
//  gram    C = X^T Y for blocked X (nbX blocks) and Y (nbY blocks).  One CTA per
//          (row chunk, bx, by) accumulates an s x s tile over its rows from shared
//          memory; partial tiles are summed over chunks in a fixed order (deterministic).
//  tsgemm  Y = beta Y + alpha X C, C of shape (nbX s) x (nbY s) row-major.  One CTA per
//          (64-row tile, output block) streams the X blocks through shared memory.
//  gram_df, tsgemm_df  the same products in pair-float arithmetic on the FP32 units: B300
//          runs FP64 at 1/64 of the FP32 rate, and at s = 32 each basis entry feeds 32
//          multiply-adds, so the FP64 kernels are bound by the FP64 pipe, not by memory.
//  colnorms ||A[:,c] - e_c B[:,c]|| for every column of a blocked set.
//  small_chol_inv / small_matmul  one-CTA Cholesky (with optional diagonal shift),
//          triangular inverse and products for n <= 256.
#include "common.cuh"
#include "pairfloat.cuh"
#include <cmath>

namespace pf {

// ------------------------------------------------------------------ gram
#define GRAM_TR 32      // rows staged per tile
#define GRAM_THREADS 256

static int gram_chunks(int64_t D, int nbX, int nbY) {
  int64_t pairs = (int64_t)nbX * nbY;
  int64_t want = ceil_div(148 * 8, pairs);
  int64_t maxc = ceil_div(D, 4 * GRAM_TR);
  int64_t c = want < maxc ? want : maxc;
  if (c < 1) c = 1;
  if (c > 65535) c = 65535;
  return (int)c;
}

// Upper bound of the partial-tile scratch for every nbX' <= nbX, nbY' <= nbY:
// chunks * pairs <= ceil(1184 / pairs) * pairs < 1184 + pairs.
size_t gram_scratch_elems(int64_t D, int s, int nbX, int nbY) {
  (void)D;
  return ((size_t)148 * 8 + (size_t)nbX * nbY) * s * s;
}

// partial[chunk][bx][by][a][b]
template <int S>
__global__ void __launch_bounds__(GRAM_THREADS) gram_partial(int64_t D, const double* __restrict__ X, int nbX,
                                                             const double* __restrict__ Y, int nbY, int64_t rows_per,
                                                             double* __restrict__ part) {
  constexpr int NOUT = S * S;
  constexpr int TPO = NOUT >= GRAM_THREADS ? 1 : GRAM_THREADS / NOUT;   // threads per output (row split)
  constexpr int OPT = NOUT >= GRAM_THREADS ? NOUT / GRAM_THREADS : 1;   // outputs per thread
  __shared__ double xs[GRAM_TR][S];
  __shared__ double ys[GRAM_TR][S];
  __shared__ double red[TPO > 1 ? GRAM_THREADS : 1];
  const int chunk = blockIdx.x, bx = blockIdx.y, by = blockIdx.z;
  const double* Xb = X + (int64_t)bx * D * S;
  const double* Yb = Y + (int64_t)by * D * S;
  const int64_t r0 = (int64_t)chunk * rows_per;
  int64_t r1 = r0 + rows_per;
  if (r1 > D) r1 = D;
  const int t = threadIdx.x;
  // output assignment
  const int o_base = (TPO > 1) ? (t % NOUT) : t;
  const int rsub = (TPO > 1) ? (t / NOUT) : 0;
  double acc[OPT];
#pragma unroll
  for (int i = 0; i < OPT; ++i) acc[i] = 0.0;
  for (int64_t rt = r0; rt < r1; rt += GRAM_TR) {
    const int nr = (int)((r1 - rt) < GRAM_TR ? (r1 - rt) : GRAM_TR);
    for (int i = t; i < GRAM_TR * S; i += GRAM_THREADS) {
      int rr = i / S, cc = i % S;
      double xv = 0.0, yv = 0.0;
      if (rr < nr) {
        xv = Xb[(rt + rr) * S + cc];
        yv = Yb[(rt + rr) * S + cc];
      }
      xs[rr][cc] = xv;
      ys[rr][cc] = yv;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < OPT; ++i) {
      const int o = o_base + i * GRAM_THREADS;
      const int a = o / S, b = o % S;
      double s = acc[i];
      for (int rr = rsub; rr < GRAM_TR; rr += TPO) s = fma(xs[rr][a], ys[rr][b], s);
      acc[i] = s;
    }
    __syncthreads();
  }
  double* P = part + (((int64_t)chunk * nbX + bx) * nbY + by) * NOUT;
  if constexpr (TPO > 1) {
    red[t] = acc[0];
    __syncthreads();
    if (t < NOUT) {
      double s = 0.0;
      for (int k = 0; k < TPO; ++k) s += red[t + k * NOUT];
      P[t] = s;
    }
  } else {
#pragma unroll
    for (int i = 0; i < OPT; ++i) P[o_base + i * GRAM_THREADS] = acc[i];
  }
}

// C[(bx*s + a) * ldc + by*s + b] = sum_chunk part[chunk][bx][by][a][b]
__global__ void gram_reduce(const double* __restrict__ part, int nchunk, int nbX, int nbY, int s, double* C, int ldc) {
  const int64_t n = (int64_t)nbX * nbY * s * s;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int c = 0; c < nchunk; ++c) acc += part[(int64_t)c * n + i];
  int64_t pair = i / (s * s);
  int ab = (int)(i % (s * s));
  int bx = (int)(pair / nbY), by = (int)(pair % nbY);
  int a = ab / s, b = ab % s;
  C[(int64_t)(bx * s + a) * ldc + by * s + b] = acc;
}

pf_status gram(int64_t D, int s, const double* X, int nbX, const double* Y, int nbY, double* C, double* scratch,
               size_t scratch_elems, cudaStream_t st) {
  if (nbX < 1 || nbY < 1) return PF_EINVAL;
  const int nchunk = gram_chunks(D, nbX, nbY);
  if ((size_t)nchunk * nbX * nbY * s * s > scratch_elems) return PF_EINVAL;
  if (nbX > 65535 || nbY > 65535) return PF_EINVAL;
  const int64_t rows_per = ceil_div(D, nchunk);
  dim3 grid(nchunk, nbX, nbY);
  switch (s) {
    case 1: gram_partial<1><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 2: gram_partial<2><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 4: gram_partial<4><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 8: gram_partial<8><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 16: gram_partial<16><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 32: gram_partial<32><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 64: gram_partial<64><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    default: return PF_EINVAL;
  }
  PF_LAUNCH_CHECK("gram_partial");
  const int64_t n = (int64_t)nbX * nbY * s * s;
  gram_reduce<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(scratch, nchunk, nbX, nbY, s, C, nbY * s);
  PF_LAUNCH_CHECK("gram_reduce");
  return PF_OK;
}

// ------------------------------------------------------------------ tsgemm
#define TS_TR 64
#define TS_THREADS 256

// Y_by[r, :] = beta Y_by[r, :] + alpha sum_bx X_bx[r, :] C[bx*S:(bx+1)*S, by*S:(by+1)*S]
template <int S>
__global__ void __launch_bounds__(TS_THREADS) tsgemm_kernel(int64_t D, const double* __restrict__ X, int nbX,
                                                            const double* __restrict__ C, int ldc, double* Y,
                                                            double alpha, double beta) {
  constexpr int NOUT = TS_TR * S;
  constexpr int OPT = NOUT / TS_THREADS > 0 ? NOUT / TS_THREADS : 1;
  extern __shared__ double ts_smem[];
  double (*xs)[S + 1] = reinterpret_cast<double (*)[S + 1]>(ts_smem);
  double (*cs)[S] = reinterpret_cast<double (*)[S]>(ts_smem + TS_TR * (S + 1));
  const int by = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * TS_TR;
  const int t = threadIdx.x;
  // thread -> (column b, rows rr = rbase + i*rstep)
  const int b = t % S;
  const int rbase = t / S;
  constexpr int RSTEP = TS_THREADS / S > 0 ? TS_THREADS / S : 1;
  const bool active = (t < S * RSTEP) && (TS_THREADS >= S || t < TS_THREADS);
  double acc[OPT];
#pragma unroll
  for (int i = 0; i < OPT; ++i) acc[i] = 0.0;
  for (int bx = 0; bx < nbX; ++bx) {
    const double* Xb = X + (int64_t)bx * D * S;
    for (int i = t; i < TS_TR * S; i += TS_THREADS) {
      int rr = i / S, cc = i % S;
      int64_t r = r0 + rr;
      xs[rr][cc] = r < D ? Xb[r * S + cc] : 0.0;
    }
    for (int i = t; i < S * S; i += TS_THREADS) {
      int a = i / S, bb = i % S;
      cs[a][bb] = C[(int64_t)(bx * S + a) * ldc + by * S + bb];
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < OPT; ++i) {
        const int rr = rbase + i * RSTEP;
        if (rr < TS_TR) {
          double s = acc[i];
#pragma unroll 8
          for (int a = 0; a < S; ++a) s = fma(xs[rr][a], cs[a][b], s);
          acc[i] = s;
        }
      }
    }
    __syncthreads();
  }
  if (active) {
    double* Yb = Y + (int64_t)by * D * S;
#pragma unroll
    for (int i = 0; i < OPT; ++i) {
      const int rr = rbase + i * RSTEP;
      const int64_t r = r0 + rr;
      if (rr < TS_TR && r < D) {
        double y = beta != 0.0 ? beta * Yb[r * S + b] : 0.0;
        Yb[r * S + b] = fma(alpha, acc[i], y);
      }
    }
  }
}

template <int S>
static pf_status launch_tsgemm(dim3 grid, cudaStream_t st, int64_t D, const double* X, int nbX, const double* C,
                               int ldc, double* Y, double alpha, double beta) {
  const int smem = (TS_TR * (S + 1) + S * S) * (int)sizeof(double);
  // set once (a function-local static initialises exactly once, thread-safely); the size is fixed per S
  static const cudaError_t attr = cudaFuncSetAttribute(tsgemm_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) { set_cuda_error(attr, "tsgemm smem attribute"); return PF_ECUDA; }
  tsgemm_kernel<S><<<grid, TS_THREADS, smem, st>>>(D, X, nbX, C, ldc, Y, alpha, beta);
  PF_LAUNCH_CHECK("tsgemm_kernel");
  return PF_OK;
}

pf_status tsgemm(int64_t D, int s, const double* X, int nbX, const double* C, int ldc, double* Y, int nbY,
                 double alpha, double beta, cudaStream_t st) {
  if (nbX < 1 || nbY < 1 || nbY > 65535) return PF_EINVAL;
  dim3 grid((unsigned)ceil_div(D, TS_TR), nbY);
  switch (s) {
    case 1: return launch_tsgemm<1>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    case 2: return launch_tsgemm<2>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    case 4: return launch_tsgemm<4>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    case 8: return launch_tsgemm<8>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    case 16: return launch_tsgemm<16>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    case 32: return launch_tsgemm<32>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    case 64: return launch_tsgemm<64>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
  }
  return PF_EINVAL;
}

// ------------------------------------------------------------------ pair-float gram / tsgemm
// Each FP64 operand is split once, while it is staged in shared memory, into hi = rn(x) and
// lo = rn(x - hi) (48 of its 53 bits).  A product accumulates by df_fma: the exact product of
// the high parts (two_prod), the cross terms hi*lo and lo*hi, and a two_sum into the running
// high part; the low parts collect in a float.  The result of a chain is the compensated dot
// product of Ogita, Rump and Oishi (2005) with operands rounded to 48 bits.

// gram_df: partial[chunk][bx][by][a][b] as in gram_partial.  256 threads as a 16 x 16 grid; a
// thread owns the T x T outputs (ta + 16 i, tb + 16 j), T = S / 16.
__device__ __forceinline__ df2 as_df(double x) { return df2(x); }
__device__ __forceinline__ df2 as_df(float2 x) { return df2(x.x, x.y); }

// TY = float2: Y given already split (hi, lo), as d2df_kernel splits it (the same pairs as
// splitting here), so a Y block shared by every bx is split once, not once per CTA.
template <int S, typename TY>
__global__ void __launch_bounds__(GRAM_THREADS) gram_df_partial(int64_t D, const double* __restrict__ X, int nbX,
                                                                const TY* __restrict__ Y, int nbY,
                                                                int64_t rows_per, double* __restrict__ part) {
  constexpr int T = S / 16;
  __shared__ df2 xs[GRAM_TR][S];
  __shared__ df2 ys[GRAM_TR][S];
  const int chunk = blockIdx.x, bx = blockIdx.y, by = blockIdx.z;
  const double* Xb = X + (int64_t)bx * D * S;
  const TY* Yb = Y + (int64_t)by * D * S;
  const int64_t r0 = (int64_t)chunk * rows_per;
  int64_t r1 = r0 + rows_per;
  if (r1 > D) r1 = D;
  const int t = threadIdx.x, ta = t / 16, tb = t % 16;
  df2 acc[T][T];
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int j = 0; j < T; ++j) acc[i][j] = df2(0.0f, 0.0f);
  for (int64_t rt = r0; rt < r1; rt += GRAM_TR) {
    const int nr = (int)((r1 - rt) < GRAM_TR ? (r1 - rt) : GRAM_TR);
    for (int i = t; i < GRAM_TR * S; i += GRAM_THREADS) {
      const int rr = i / S, cc = i % S;
      double xv = 0.0;
      TY yv{};
      if (rr < nr) {
        xv = Xb[(rt + rr) * S + cc];
        yv = Yb[(rt + rr) * S + cc];
      }
      xs[rr][cc] = df2(xv);
      ys[rr][cc] = as_df(yv);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < GRAM_TR; ++rr) {
      df2 xv[T], yv[T];
#pragma unroll
      for (int i = 0; i < T; ++i) xv[i] = xs[rr][ta + 16 * i];
#pragma unroll
      for (int j = 0; j < T; ++j) yv[j] = ys[rr][tb + 16 * j];
#pragma unroll
      for (int i = 0; i < T; ++i)
#pragma unroll
        for (int j = 0; j < T; ++j) acc[i][j] = df_fma(xv[i], yv[j], acc[i][j]);
    }
    __syncthreads();
  }
  double* P = part + (((int64_t)chunk * nbX + bx) * nbY + by) * (S * S);
#pragma unroll
  for (int i = 0; i < T; ++i)
#pragma unroll
    for (int j = 0; j < T; ++j) P[(ta + 16 * i) * S + tb + 16 * j] = (double)acc[i][j].hi + (double)acc[i][j].lo;
}

template <typename TY>
static pf_status gram_df_any(int64_t D, int s, const double* X, int nbX, const TY* Y, int nbY, double* C,
                             double* scratch, size_t scratch_elems, cudaStream_t st) {
  if (nbX < 1 || nbY < 1) return PF_EINVAL;
  const int nchunk = gram_chunks(D, nbX, nbY);
  if ((size_t)nchunk * nbX * nbY * s * s > scratch_elems) return PF_EINVAL;
  if (nbX > 65535 || nbY > 65535) return PF_EINVAL;
  const int64_t rows_per = ceil_div(D, nchunk);
  dim3 grid(nchunk, nbX, nbY);
  switch (s) {
    case 16: gram_df_partial<16, TY><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 32: gram_df_partial<32, TY><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    case 64: gram_df_partial<64, TY><<<grid, GRAM_THREADS, 0, st>>>(D, X, nbX, Y, nbY, rows_per, scratch); break;
    default: return PF_EINVAL;
  }
  PF_LAUNCH_CHECK("gram_df_partial");
  const int64_t n = (int64_t)nbX * nbY * s * s;
  gram_reduce<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(scratch, nchunk, nbX, nbY, s, C, nbY * s);
  PF_LAUNCH_CHECK("gram_reduce");
  return PF_OK;
}

pf_status gram_df(int64_t D, int s, const double* X, int nbX, const double* Y, int nbY, double* C, double* scratch,
                  size_t scratch_elems, cudaStream_t st) {
  if (s != 16 && s != 32 && s != 64) return gram(D, s, X, nbX, Y, nbY, C, scratch, scratch_elems, st);
  return gram_df_any<double>(D, s, X, nbX, Y, nbY, C, scratch, scratch_elems, st);
}

pf_status gram_df_ysplit(int64_t D, int s, const double* X, int nbX, const float2* Y, int nbY, double* C,
                         double* scratch, size_t scratch_elems, cudaStream_t st) {
  return gram_df_any<float2>(D, s, X, nbX, Y, nbY, C, scratch, scratch_elems, st);
}

// tsgemm_df: one CTA per (64-row tile, output block) as in tsgemm_kernel; thread t owns column
// b = t % S of the rows t / S + i (256 / S).
template <int S>
__global__ void __launch_bounds__(TS_THREADS) tsgemm_df_kernel(int64_t D, const double* __restrict__ X, int nbX,
                                                               const double* __restrict__ C, int ldc, double* Y,
                                                               double alpha, double beta) {
  constexpr int RSTEP = TS_THREADS / S;
  constexpr int OPT = TS_TR / RSTEP;
  extern __shared__ df2 tsd_smem[];
  df2 (*xs)[S] = reinterpret_cast<df2 (*)[S]>(tsd_smem);
  df2 (*cs)[S] = reinterpret_cast<df2 (*)[S]>(tsd_smem + TS_TR * S);
  const int by = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * TS_TR;
  const int t = threadIdx.x;
  const int b = t % S, rbase = t / S;
  df2 acc[OPT];
#pragma unroll
  for (int i = 0; i < OPT; ++i) acc[i] = df2(0.0f, 0.0f);
  for (int bx = 0; bx < nbX; ++bx) {
    const double* Xb = X + (int64_t)bx * D * S;
    for (int i = t; i < TS_TR * S; i += TS_THREADS) {
      const int rr = i / S, cc = i % S;
      const int64_t r = r0 + rr;
      xs[rr][cc] = df2(r < D ? Xb[r * S + cc] : 0.0);
    }
    for (int i = t; i < S * S; i += TS_THREADS) {
      const int a = i / S, bb = i % S;
      cs[a][bb] = df2(C[(int64_t)(bx * S + a) * ldc + by * S + bb]);
    }
    __syncthreads();
#pragma unroll 4
    for (int a = 0; a < S; ++a) {
      const df2 c = cs[a][b];
#pragma unroll
      for (int i = 0; i < OPT; ++i) acc[i] = df_fma(xs[rbase + i * RSTEP][a], c, acc[i]);
    }
    __syncthreads();
  }
  double* Yb = Y + (int64_t)by * D * S;
#pragma unroll
  for (int i = 0; i < OPT; ++i) {
    const int64_t r = r0 + rbase + i * RSTEP;
    if (r < D) {
      const double y = beta != 0.0 ? beta * Yb[r * S + b] : 0.0;
      Yb[r * S + b] = fma(alpha, (double)acc[i].hi + (double)acc[i].lo, y);
    }
  }
}

template <int S>
static pf_status launch_tsgemm_df(dim3 grid, cudaStream_t st, int64_t D, const double* X, int nbX, const double* C,
                                  int ldc, double* Y, double alpha, double beta) {
  const int smem = (TS_TR * S + S * S) * (int)sizeof(df2);
  // set once, as in launch_tsgemm
  static const cudaError_t attr = cudaFuncSetAttribute(tsgemm_df_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (attr != cudaSuccess) { set_cuda_error(attr, "tsgemm_df smem attribute"); return PF_ECUDA; }
  tsgemm_df_kernel<S><<<grid, TS_THREADS, smem, st>>>(D, X, nbX, C, ldc, Y, alpha, beta);
  PF_LAUNCH_CHECK("tsgemm_df_kernel");
  return PF_OK;
}

pf_status tsgemm_df(int64_t D, int s, const double* X, int nbX, const double* C, int ldc, double* Y, int nbY,
                    double alpha, double beta, cudaStream_t st) {
  if (s != 16 && s != 32 && s != 64) return tsgemm(D, s, X, nbX, C, ldc, Y, nbY, alpha, beta, st);
  if (nbX < 1 || nbY < 1 || nbY > 65535) return PF_EINVAL;
  dim3 grid((unsigned)ceil_div(D, TS_TR), nbY);
  switch (s) {
    case 16: return launch_tsgemm_df<16>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    case 32: return launch_tsgemm_df<32>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
    default: return launch_tsgemm_df<64>(grid, st, D, X, nbX, C, ldc, Y, alpha, beta);
  }
}

// ------------------------------------------------------------------ column norms
// part[chunk][col] = sum over the chunk's rows of (A - e B)^2
__global__ void colnorm_partial(int64_t D, int s, const double* __restrict__ A, const double* __restrict__ B,
                                const double* __restrict__ e, int64_t rows_per, double* part) {
  const int blk = blockIdx.y, chunk = blockIdx.x;
  const int ncol = s;
  const double* Ab = A + (int64_t)blk * D * s;
  const double* Bb = B ? B + (int64_t)blk * D * s : nullptr;
  const int64_t r0 = (int64_t)chunk * rows_per;
  int64_t r1 = r0 + rows_per;
  if (r1 > D) r1 = D;
  __shared__ double sh[256];
  // thread t handles column t % s, rows r0 + t/s, stepping by 256/s (s <= 64 divides 256)
  const int c = threadIdx.x % ncol;
  const int rstep = blockDim.x / ncol;
  const double ec = (B && e) ? e[blk * s + c] : 0.0;
  double acc = 0.0;
  for (int64_t r = r0 + threadIdx.x / ncol; r < r1; r += rstep) {
    double x = Ab[r * s + c];
    if (Bb) x -= ec * Bb[r * s + c];
    acc = fma(x, x, acc);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < ncol) {
    double t = 0.0;
    for (int k = 0; k < rstep; ++k) t += sh[threadIdx.x + k * ncol];
    part[((int64_t)chunk * gridDim.y + blk) * s + threadIdx.x] = t;
  }
}

__global__ void colnorm_final(const double* part, int nchunk, int ncols, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncols) return;
  double t = 0.0;
  for (int c = 0; c < nchunk; ++c) t += part[(int64_t)c * ncols + i];
  out[i] = sqrt(t);
}

pf_status colnorms(int64_t D, int s, const double* A, const double* B, const double* e, int nb, double* norms,
                   double* scratch, size_t scratch_elems, cudaStream_t st) {
  int nchunk = (int)ceil_div(D, 4096);
  if (nchunk > 256) nchunk = 256;
  if ((size_t)nchunk * nb * s > scratch_elems) return PF_EINVAL;
  const int64_t rows_per = ceil_div(D, nchunk);
  colnorm_partial<<<dim3(nchunk, nb), 256, 0, st>>>(D, s, A, B, e, rows_per, scratch);
  PF_LAUNCH_CHECK("colnorm_partial");
  colnorm_final<<<(unsigned)ceil_div(nb * s, 128), 128, 0, st>>>(scratch, nchunk, nb * s, norms);
  PF_LAUNCH_CHECK("colnorm_final");
  return PF_OK;
}

// ------------------------------------------------------------------ conversions
__global__ void d2f_kernel(const double* x, float* y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
__global__ void f2d_kernel(const float* x, double* y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}
pf_status convert_d2f(const double* x, float* y, int64_t n, cudaStream_t st) {
  d2f_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(x, y, n);
  PF_LAUNCH_CHECK("d2f_kernel");
  return PF_OK;
}
pf_status convert_f2d(const float* x, double* y, int64_t n, cudaStream_t st) {
  f2d_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(x, y, n);
  PF_LAUNCH_CHECK("f2d_kernel");
  return PF_OK;
}
// In place allowed: each thread reads its 8 bytes before writing them.
__global__ void d2df_kernel(const double* x, float2* y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const double v = x[i];
    const float hi = (float)v;
    y[i] = make_float2(hi, (float)(v - (double)hi));
  }
}
__global__ void df2d_kernel(const float2* x, double* y, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const float2 v = x[i];
    y[i] = (double)v.x + (double)v.y;   // exact: the pair's sum has at most 49 significant bits
  }
}
pf_status convert_d2df(const double* x, float2* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return PF_OK;
  d2df_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(x, y, n);
  PF_LAUNCH_CHECK("d2df_kernel");
  return PF_OK;
}
pf_status convert_df2d(const float2* x, double* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return PF_OK;
  df2d_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(x, y, n);
  PF_LAUNCH_CHECK("df2d_kernel");
  return PF_OK;
}

// ------------------------------------------------------------------ small dense (one CTA)
// G row-major n x n (symmetric).  R upper with (G + shift I) = R^T R, shift = shift_rel * trace(G),
// factored in place in R (global memory; n <= 512 keeps it in L2).  Rinv = R^{-1}.
// status[0] = 1 if a pivot is not positive (the factor is then not usable).
__global__ void small_chol_inv_kernel(const double* G, int n, double shift_rel, double* R, double* Rinv, int* status) {
  __shared__ double tr_sh[32];
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  double tr = 0.0;
  for (int i = t; i < n; i += blockDim.x) tr += G[i * n + i];
  tr = block_sum(tr, tr_sh);
  const double shift = shift_rel * tr;
  for (int i = t; i < n * n; i += blockDim.x) {
    int r = i / n, c = i % n;
    double g = 0.5 * (G[r * n + c] + G[c * n + r]);
    R[i] = (c >= r) ? g + (r == c ? shift : 0.0) : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      double d = R[k * n + k];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1.0;
      }
      R[k * n + k] = sqrt(d);
    }
    __syncthreads();
    const double pk = R[k * n + k];
    for (int j = k + 1 + t; j < n; j += blockDim.x) R[k * n + j] /= pk;
    __syncthreads();
    const int m = n - k - 1;
    for (int i = t; i < m * m; i += blockDim.x) {
      int r = k + 1 + i / m, c = k + 1 + i % m;
      if (c >= r) R[r * n + c] -= R[k * n + r] * R[k * n + c];
    }
    __syncthreads();
  }
  for (int c = t; c < n; c += blockDim.x) {
    for (int r = n - 1; r >= 0; --r) {
      double v = (r == c) ? 1.0 : 0.0;
      for (int k = r + 1; k <= c; ++k) v -= R[r * n + k] * Rinv[k * n + c];
      Rinv[r * n + c] = (r <= c) ? v / R[r * n + r] : 0.0;
    }
  }
  if (t == 0) status[0] = bad;
}

// The same factorisation for n <= 64 with the matrix in shared memory.  Cholesky, right-looking: per
// pivot k one thread forms r_kk = sqrt(a_kk) and its reciprocal, the trailing upper triangle takes
// a_rc -= (a_kr / r_kk)(a_kc / r_kk) with the reciprocal, then row k is scaled.  The inverse X of the
// upper-triangular R by rows from the bottom: once row k of X is final every row i < k takes
// x_ic -= r_ik x_kc (c >= k), and row k - 1, final after that, is scaled by 1 / r_{k-1,k-1} in the same
// pass, so one barrier per row remains.  The global-memory kernel above spent ~80 us at n = 32 on its
// three barriers per pivot with every operand in L1 and its one-thread-per-column back substitution.
#define PF_CHOL_SM_N 64
__global__ void __launch_bounds__(256) small_chol_inv_sm_kernel(const double* G, int n, double shift_rel, double* R,
                                                                double* Rinv, int* status) {
  extern __shared__ __align__(16) double smc[];
  __shared__ double tr_sh[32];
  __shared__ int bad;
  const int ld = n + 1;
  double* A = smc;              // n x ld, row-major: the upper triangle becomes R
  double* X = A + n * ld;       // R^{-1}
  double* rdg = X + n * ld;     // 1 / r_kk
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  double tr = 0.0;
  for (int i = t; i < n; i += blockDim.x) tr += G[i * n + i];
  tr = block_sum(tr, tr_sh);
  const double shift = shift_rel * tr;
  for (int i = t; i < n * n; i += blockDim.x) {
    const int r = i / n, c = i % n;
    A[r * ld + c] = c >= r ? 0.5 * (G[r * n + c] + G[c * n + r]) + (r == c ? shift : 0.0) : 0.0;
    X[r * ld + c] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      double dk = A[k * ld + k];
      if (!(dk > 0.0)) {
        bad = 1;
        dk = 1.0;
      }
      const double pk = sqrt(dk);
      A[k * ld + k] = pk;
      rdg[k] = 1.0 / pk;
    }
    __syncthreads();
    const double rp = rdg[k];
    const int m = n - k - 1;
    for (int i = t; i < m * m; i += blockDim.x) {
      const int r = k + 1 + i / m, c = k + 1 + i % m;
      if (c >= r) A[r * ld + c] -= (A[k * ld + r] * rp) * (A[k * ld + c] * rp);
    }
    __syncthreads();
    for (int j = k + 1 + t; j < n; j += blockDim.x) A[k * ld + j] *= rp;   // row k is read again only below
  }
  if (t == 0) X[(n - 1) * ld + n - 1] = rdg[n - 1];
  __syncthreads();
  for (int k = n - 1; k >= 1; --k) {
    const int w = n - k;   // columns k..n-1
    for (int i = t; i < k * w; i += blockDim.x) {
      const int r = i / w, c = k + i % w;
      double x = X[r * ld + c] - A[r * ld + k] * X[k * ld + c];
      if (r == k - 1) x *= rdg[k - 1];
      X[r * ld + c] = x;
    }
    if (t == 0) X[(k - 1) * ld + k - 1] = rdg[k - 1];
    __syncthreads();
  }
  for (int i = t; i < n * n; i += blockDim.x) {
    const int r = i / n, c = i % n;
    R[i] = c >= r ? A[r * ld + c] : 0.0;
    Rinv[i] = c >= r ? X[r * ld + c] : 0.0;
  }
  if (t == 0) status[0] = bad;
}

pf_status small_chol_inv(const double* G, int n, double shift_rel, double* R, double* Rinv, int* status,
                         cudaStream_t st) {
  if (n < 1 || n > 512) return PF_EINVAL;
  if (n <= PF_CHOL_SM_N) {
    static const cudaError_t attr = cudaFuncSetAttribute(
        small_chol_inv_sm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)((2 * PF_CHOL_SM_N * (PF_CHOL_SM_N + 1) + PF_CHOL_SM_N) * sizeof(double)));
    PF_CUDA(attr);
    const size_t smem = (size_t)(2 * n * (n + 1) + n) * sizeof(double);
    small_chol_inv_sm_kernel<<<1, 256, smem, st>>>(G, n, shift_rel, R, Rinv, status);
    PF_LAUNCH_CHECK("small_chol_inv_sm_kernel");
    return PF_OK;
  }
  small_chol_inv_kernel<<<1, 512, 0, st>>>(G, n, shift_rel, R, Rinv, status);
  PF_LAUNCH_CHECK("small_chol_inv_kernel");
  return PF_OK;
}

__global__ void small_matmul_kernel(const double* A, const double* B, double* C, int n) {
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    int r = i / n, c = i % n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = fma(A[r * n + k], B[k * n + c], s);
    C[i] = s;
  }
}

pf_status small_matmul(const double* A, const double* B, double* C, int n, cudaStream_t st) {
  small_matmul_kernel<<<1, 256, 0, st>>>(A, B, C, n);
  PF_LAUNCH_CHECK("small_matmul_kernel");
  return PF_OK;
}

}  // namespace pf
