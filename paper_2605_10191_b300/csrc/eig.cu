// Symmetric eigensolver for the projected (Lanczos) matrix H_L, FP64, on the device.
//
// Used by the convergence checks (Eq. blocklan_criterion needs eigenvectors t_j of H_L)
// and by the Rayleigh-Ritz steps.  Only selected eigenpairs are computed:
//   1. Householder tridiagonalisation A = Q T Q^T (reflectors kept in A's columns): one
//      thread-block-cluster launch with the matrix in distributed shared memory for orders up to
//      ~620, up to 3000 two launches per column over the whole GPU (reflector, p = tau A22 v and
//      w = p - (tau/2)(p.v) v; the rank-2 update A22 -= v w^T + w v^T of the full trailing block),
//      above that four.
//   2. Multisection with Sturm counts for each requested index (one warp, in a CTA of its
//      own, per index).
//   3. Inverse iteration on T - lambda I (tridiagonal LU with partial pivoting), one
//      CTA per cluster of eigenvalues closer than 1e-6 ||T||; members of a cluster are kept
//      orthogonal by modified Gram-Schmidt against the earlier members.
//   4. Back-transformation z = H_0 H_1 ... H_{n-3} y, one CTA per eigenvector.
#include "common.cuh"
#include "pairfloat.cuh"
#include <cooperative_groups.h>
#include <cmath>
#include <map>
#include <mutex>
#include <algorithm>

namespace pf {

struct EigLayout {
  size_t aw, d, e, tau, p, w, y, lu, cl, sturm, ticket, total;
};

static EigLayout eig_layout(int n, int q) {
  EigLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += (bytes + 255) & ~(size_t)255; return r; };
  L.aw = take((size_t)n * n * 8);
  L.d = take((size_t)n * 8);
  L.e = take((size_t)n * 8);
  L.tau = take((size_t)n * 8);
  L.p = take((size_t)3 * n * 8);   // p, w, v of the two-launch column step
  L.w = take((size_t)q * 8);
  L.y = take((size_t)n * q * 8);
  L.lu = take((size_t)q * 6 * n * 8);
  L.cl = take((size_t)(q + 2) * 4 * 2);
  L.sturm = take((size_t)n * 32);   // e^2 (FP64), d and e^2 scaled (FP32 and pair-float)
  L.ticket = take(16);
  L.total = o;
  return L;
}

size_t eig_workspace_bytes(int nmax, int qmax) { return eig_layout(nmax, qmax).total; }

// A kernel's dynamic shared-memory limit is one value per kernel and device, shared by every host
// thread.  Setting it to each call's own size lets a thread that lowers it (a smaller matrix) break
// another thread's launch of a larger one in between; calls on distinct handles may run on different
// threads.  This raises the limit to `bytes` when it is lower, never lowers it, and leaves sizes up to
// the default 48 KB alone.
static pf_status raise_smem_limit(const void* kern, size_t bytes) {
  if (bytes <= (size_t)48 * 1024) return PF_OK;
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[std::make_pair(kern, dev)];
  if (bytes <= cur) return PF_OK;
  PF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return PF_OK;
}

// One entry of the rank-2 update A22 -= v w^T + w v^T (row l, column c), as two FMAs; every form of
// the tridiagonalisation calls this one expression.
__device__ __forceinline__ double rank2_entry(double a, double vl, double wc, double wl, double vc) {
  return fma(-vl, wc, fma(-wl, vc, a));
}

// Deterministic block sum over blockDim.x threads of which only the first nact can hold a nonzero
// term: warps beyond them skip their shuffle tree (their partial is +0, as block_sum would find), so the
// result is block_sum's, bit for bit, without the idle warps' FP64 additions on the SM's slow FP64 pipe.
__device__ double block_sum_act(double v, double* sh, int nact) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w < ((nact + 31) >> 5)) v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  double r = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// Householder reflector of x (alpha = x_0, sig = sum_{i>=1} x_i^2): H x = beta e_0, H = I - tau v v^T with
// v = x / (alpha - beta), v_0 = 1 (scale = 1 / (alpha - beta)).  Thread 0 evaluates the square root and
// the two divisions and the block reads them from shared memory (rf, 3 doubles; the caller's next write
// to rf follows a barrier): on B300 a division is ~1000 cycles of dependent FP64 operations, and every
// warp of a 512-thread CTA evaluating them kept the SM's FP64 pipe busy for ~7000 cycles per column.
struct Refl {
  double beta, t, scale;
};
__device__ Refl reflector(double alpha, double sig, double* rf) {
  if (threadIdx.x == 0) {
    double beta, t, scale;
    if (sig == 0.0) {
      beta = alpha;
      t = 0.0;
      scale = 0.0;
    } else {
      const double nrm = sqrt(alpha * alpha + sig);
      beta = alpha <= 0.0 ? nrm : -nrm;
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    rf[0] = beta;
    rf[1] = t;
    rf[2] = scale;
  }
  __syncthreads();
  return Refl{rf[0], rf[1], rf[2]};
}

// Aw (column-major n x n) = A (row-major, lda); A is symmetric.
__global__ void eig_copy_kernel(const double* A, int lda, int n, double* Aw) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)n * n) return;
  int c = (int)(i / n), r = (int)(i % n);
  Aw[i] = 0.5 * (A[(int64_t)r * lda + c] + A[(int64_t)c * lda + r]);
}

// Reflector for column j: x = Aw[j+1.., j].  H x = beta e1, H = I - tau v v^T, v_0 = 1.
__global__ void house_kernel(double* Aw, int n, int j, double* d, double* e, double* tau) {
  __shared__ double sh[32];
  __shared__ double rf[3];
  const int m = n - j - 1;
  double* x = Aw + (int64_t)j * n + j + 1;
  double sig = 0.0;
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) sig += x[i] * x[i];
  sig = block_sum_act(sig, sh, m - 1);
  const Refl rfl = reflector(x[0], sig, rf);
  const double beta = rfl.beta, t = rfl.t, scale = rfl.scale;
  __syncthreads();
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) x[i] *= scale;
  if (threadIdx.x == 0) {
    x[0] = 1.0;
    d[j] = Aw[(int64_t)j * n + j];
    e[j] = beta;
    tau[j] = t;
  }
}

// p_i = tau_j * sum_l A22[l, i] v_l, i < m.  One warp per i (column i of A22 is contiguous).
__global__ void symv_kernel(const double* Aw, int n, int j, const double* tau, double* p) {
  const int m = n - j - 1;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= m) return;
  const double* v = Aw + (int64_t)j * n + j + 1;
  const double* col = Aw + (int64_t)(j + 1 + warp) * n + j + 1;
  double s = 0.0;
  for (int l = lane; l < m; l += 32) s = fma(col[l], v[l], s);
  s = warp_sum(s);
  if (lane == 0) p[warp] = tau[j] * s;
}

// w = p - (tau/2)(p.v) v, written to p + n (one CTA).
__global__ void wvec_kernel(const double* Aw, int n, int j, const double* tau, double* p) {
  __shared__ double sh[32];
  const int m = n - j - 1;
  const double* v = Aw + (int64_t)j * n + j + 1;
  double g = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) g = fma(p[i], v[i], g);
  g = block_sum_act(g, sh, m);
  const double c = 0.5 * tau[j] * g;
  for (int i = threadIdx.x; i < m; i += blockDim.x) p[n + i] = p[i] - c * v[i];
}

// A22[l, i] -= v_l w_i + w_l v_i over the full trailing block.
__global__ void rank2_kernel(double* Aw, int n, int j, const double* p) {
  const int m = n - j - 1;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int i = (int)(idx / m), l = (int)(idx % m);
  const double* v = Aw + (int64_t)j * n + j + 1;
  const double* w = p + n;
  double* a = Aw + (int64_t)(j + 1 + i) * n + j + 1 + l;
  *a = rank2_entry(*a, v[l], w[i], w[l], v[i]);
}

// The same column step in two launches, for orders above the distributed-shared-memory kernel's
// reach (to n = 3000: v and w of a column in 48 KB of shared memory), with the arithmetic of house/symv/wvec/rank2_kernel operation for operation (the same bits).
// house_symv_kernel(j): every CTA forms the reflector of column j itself (the same block sum as
// house_kernel, so the same bits in every CTA) and v = x * scale (v_0 = 1) in shared memory, its warps
// form p_i = tau A22[:, i] . v, and CTA 0 stores d, e, tau.  The CTA that finishes last (a ticket taken
// after a fence; no CTA waits for another) forms g = p . v (wvec_kernel's block sum) and
// w = p - (tau/2) g v, and stores v and w.  rank2_vw_kernel(j): every CTA stages v and w in shared
// memory and applies the rank-2 update to its part of A22; CTA 0 stores v into column j for the
// back-transformation (no launch reads column j after house_symv_kernel(j)).  Per update entry two
// FMAs: the previous form rebuilt v and w from x in every entry, six FP64 operations.
__global__ void house_symv_kernel(double* Aw, int n, int j, double* d, double* e, double* tau, double* p,
                                  unsigned* ticket) {
  extern __shared__ __align__(16) double vs[];   // v, m entries
  __shared__ double sh[32];
  __shared__ double rf[3];
  __shared__ unsigned last;
  const int m = n - j - 1;
  const double* x = Aw + (int64_t)j * n + j + 1;
  double sig = 0.0;
  for (int i = 1 + threadIdx.x; i < m; i += blockDim.x) sig += x[i] * x[i];
  sig = block_sum_act(sig, sh, m - 1);
  const Refl rfl = reflector(x[0], sig, rf);
  const double beta = rfl.beta, t = rfl.t, scale = rfl.scale;
  for (int l = threadIdx.x; l < m; l += blockDim.x) vs[l] = l == 0 ? 1.0 : x[l] * scale;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d[j] = Aw[(int64_t)j * n + j];
    e[j] = beta;
    tau[j] = t;
  }
  __syncthreads();
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp < m) {
    const double* col = Aw + (int64_t)(j + 1 + warp) * n + j + 1;
    double s = 0.0;
    for (int l = lane; l < m; l += 32) s = fma(col[l], vs[l], s);
    s = warp_sum(s);
    if (lane == 0) p[warp] = t * s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!last) return;
  __threadfence();
  double g = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) g = fma(__ldcg(p + i), vs[i], g);
  g = block_sum_act(g, sh, m);
  if (threadIdx.x == 0) rf[0] = 0.5 * t * g;
  __syncthreads();
  const double c = rf[0];
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    p[n + i] = __ldcg(p + i) - c * vs[i];
    p[2 * n + i] = vs[i];
  }
  if (threadIdx.x == 0) *ticket = 0u;   // for the next column's launch
}

__global__ void rank2_vw_kernel(double* Aw, int n, int j, const double* p) {
  extern __shared__ __align__(16) double vw[];   // v (m), then w (m)
  const int m = n - j - 1;
  double* vv = vw;
  double* ww = vw + m;
  for (int l = threadIdx.x; l < m; l += blockDim.x) {
    vv[l] = p[2 * n + l];
    ww[l] = p[n + l];
  }
  __syncthreads();
  if (blockIdx.x == 0) {   // column j's stored reflector, v_0 = 1
    double* x = Aw + (int64_t)j * n + j + 1;
    for (int l = threadIdx.x; l < m; l += blockDim.x) x[l] = vv[l];
  }
  // grid-stride over the m x m entries (m^2 < 2^31 for the orders this form takes)
  const int tot = m * m;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < tot; idx += gridDim.x * blockDim.x) {
    const int i = idx / m, l = idx - i * m;
    double* a = Aw + (int64_t)(j + 1 + i) * n + j + 1 + l;
    *a = rank2_entry(*a, vv[l], ww[i], ww[l], vv[i]);
  }
}

// The whole tridiagonalisation in one launch: one thread-block cluster of CS CTAs walks the
// columns and meets at the hardware cluster barrier (arrive.release / wait.acquire) between
// the four phases of each column: the reflector (CTA 0, as house_kernel), p = tau A22 v (warps
// of the whole cluster, as symv_kernel), w = p - (tau/2)(p.v) v (every CTA forms the dot in the
// same order, then writes its slice, as wvec_kernel) and the rank-2 update (as rank2_kernel).
// Data another CTA wrote is read with L2-only loads.  One launch instead of four per column; it is
// now the fallback (n <= 400) where the distributed-shared-memory form below cannot be launched.
// No spin-waits: the barriers are hardware barriers.
#define PF_TRI_NT 512
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(PF_TRI_NT) tridiag_cluster_kernel(double* Aw, int n, double* d, double* e,
                                                                    double* tau, double* p) {
  __shared__ double sh[32];
  __shared__ double rf[3];
  unsigned rank, cs;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(cs));
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int gwarp = (int)rank * (PF_TRI_NT / 32) + warp, nwarps = (int)cs * (PF_TRI_NT / 32);
  const int gtid = (int)rank * PF_TRI_NT + tid, nthr = (int)cs * PF_TRI_NT;
  (void)nthr;
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    double* x = Aw + (int64_t)j * n + j + 1;
    if (rank == 0) {   // reflector: H x = beta e1, H = I - tau v v^T, v_0 = 1
      double sig = 0.0;
      for (int i = 1 + tid; i < m; i += PF_TRI_NT) {
        const double xi = ldcg(x + i);
        sig += xi * xi;
      }
      sig = block_sum_act(sig, sh, m - 1);
      const Refl rfl = reflector(ldcg(x), sig, rf);
      const double beta = rfl.beta, t = rfl.t, scale = rfl.scale;
      __syncthreads();
      for (int i = 1 + tid; i < m; i += PF_TRI_NT) x[i] = ldcg(x + i) * scale;
      if (tid == 0) {
        x[0] = 1.0;
        d[j] = ldcg(Aw + (int64_t)j * n + j);
        e[j] = beta;
        tau[j] = t;
      }
    }
    cluster_sync_all();
    const double tj = ldcg(tau + j);
    // p_i = tau_j sum_l A22[l, i] v_l
    for (int i = gwarp; i < m; i += nwarps) {
      const double* col = Aw + (int64_t)(j + 1 + i) * n + j + 1;
      double sacc = 0.0;
      for (int l = lane; l < m; l += 32) sacc = fma(ldcg(col + l), ldcg(x + l), sacc);
      sacc = warp_sum(sacc);
      if (lane == 0) p[i] = tj * sacc;
    }
    cluster_sync_all();
    // w = p - (tau/2)(p.v) v
    double g = 0.0;
    for (int i = tid; i < m; i += PF_TRI_NT) g = fma(ldcg(p + i), ldcg(x + i), g);
    g = block_sum_act(g, sh, m);
    const double c = 0.5 * tj * g;
    for (int i = gtid; i < m; i += nthr) p[n + i] = ldcg(p + i) - c * ldcg(x + i);
    cluster_sync_all();
    // A22[l, i] -= v_l w_i + w_l v_i
    const double* w = p + n;
    for (int i = gwarp; i < m; i += nwarps) {   // column i of A22 per warp, rows across the lanes
      double* col = Aw + (int64_t)(j + 1 + i) * n + j + 1;
      const double wi = ldcg(w + i), vi = ldcg(x + i);
      for (int l = lane; l < m; l += 32) col[l] = rank2_entry(ldcg(col + l), ldcg(x + l), wi, ldcg(w + l), vi);
    }
    cluster_sync_all();
  }
}

// The tridiagonalisation for small orders in one thread-block cluster with the matrix in distributed
// shared memory, one cluster barrier per column.  Column c lives in the shared memory of CTA c mod cs
// (its k-th column, k = c / cs), for the whole reduction.  Every CTA also holds its own copy of the
// column being reduced.  Per column j:
//   1. every CTA forms the reflector of column j from its copy (the same block sum and operations as
//      house_kernel, so the same bits in every CTA); CTA 0 stores d, e, tau, and the owner of column
//      j keeps v in its stored column for the back-transformation;
//   2. every CTA forms p_c = tau A22[:, c] . v for its own columns c > j and stores each p_c into
//      every CTA's p buffer; the owner of column j + 1 stores that column into every CTA's copy
//      buffer;
//   -- cluster barrier --
//   3. every CTA forms g = p . v and w = p - (tau/2) g v and applies the rank-2 update
//      A22 -= v w^T + w v^T to its own columns and to its copy of column j + 1 (the same expression,
//      so the copy equals the owner's column bit for bit).
// The p and copy buffers alternate between two halves by the parity of j: a CTA that has passed
// column j's barrier writes the other half, which every CTA finished reading before it arrived at
// that barrier.  The result is the tridiagonal of house/symv/wvec/rank2_kernel, bit for bit.  The
// barriers are hardware barriers (no spin-waits); remote shared memory is written only between the
// first and the last barrier, while every CTA of the cluster is resident.
#define PF_TRI_DS_NT 512
__global__ void __launch_bounds__(PF_TRI_DS_NT) tridiag_dsmem_kernel(double* Aw, int n, int ldc, double* d, double* e,
                                                                   double* tau) {
  extern __shared__ __align__(16) double ds[];
  __shared__ double sh[32];
  __shared__ double rf[3];
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank(), cs = cl.num_blocks();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  double* cols = ds;                                 // ldc columns of n: column k*cs + rank at cols + k*n
  double* vb = cols + (size_t)ldc * n;               // v, indexed by absolute row
  double* wb = vb + n;                               // w
  double* pb = wb + n;                               // p of column j in pb + (j & 1) * n (every CTA's stores)
  double* xb = pb + 2 * (size_t)n;                   // column j of the partly reduced matrix in xb + (j & 1) * n
  for (int k = 0; k < ldc; ++k) {
    const int c = k * (int)cs + (int)rank;
    if (c < n)
      for (int r = tid; r < n; r += PF_TRI_DS_NT) cols[(size_t)k * n + r] = Aw[(int64_t)c * n + r];
  }
  for (int r = tid; r < n; r += PF_TRI_DS_NT) xb[r] = Aw[r];
  __syncthreads();
  cluster_sync_all();
  for (int j = 0; j + 2 < n; ++j) {
    const int m = n - j - 1;
    const double* xc = xb + (size_t)(j & 1) * n;
    // 1. reflector: H x = beta e1, H = I - tau v v^T, v_0 = 1, x = rows j+1.. of column j
    double sig = 0.0;
    for (int i = 1 + tid; i < m; i += PF_TRI_DS_NT) sig += xc[j + 1 + i] * xc[j + 1 + i];
    sig = block_sum_act(sig, sh, m - 1);
    const Refl rfl = reflector(xc[j + 1], sig, rf);
    const double beta = rfl.beta, t = rfl.t, scale = rfl.scale;
    for (int i = 1 + tid; i < m; i += PF_TRI_DS_NT) vb[j + 1 + i] = xc[j + 1 + i] * scale;
    if (tid == 0) {
      vb[j + 1] = 1.0;
      if (rank == 0) {
        d[j] = xc[j];
        e[j] = beta;
        tau[j] = t;
      }
    }
    __syncthreads();
    if (rank == (unsigned)(j % (int)cs)) {
      double* own = cols + (size_t)(j / (int)cs) * n;
      for (int i = tid; i < m; i += PF_TRI_DS_NT) own[j + 1 + i] = vb[j + 1 + i];
    }
    // 2. p_c for the own columns c > j: one warp per column, the product stored into every CTA
    double* pj = pb + (size_t)(j & 1) * n;
    const int k0 = (j + 1 - (int)rank + (int)cs - 1) / (int)cs;   // first own column index with c > j
    for (int k = k0 + warp; k < ldc; k += PF_TRI_DS_NT / 32) {
      const int c = k * (int)cs + (int)rank;
      if (c >= n) break;
      const double* col = cols + (size_t)k * n;
      double acc = 0.0;
      for (int l = j + 1 + lane; l < n; l += 32) acc = fma(col[l], vb[l], acc);
      acc = warp_sum(acc);
      if (lane < (int)cs) *cl.map_shared_rank(pj + c, (unsigned)lane) = t * acc;
    }
    // the owner of column j + 1 hands its rows j+1.. to every CTA (the next reflector's input)
    if (j + 3 < n && rank == (unsigned)((j + 1) % (int)cs)) {
      const double* own = cols + (size_t)((j + 1) / (int)cs) * n;
      double* dst = xb + (size_t)((j + 1) & 1) * n;
      for (int i = tid; i < m * (int)cs; i += PF_TRI_DS_NT) {
        const int r = i / m, row = j + 1 + i % m;
        *cl.map_shared_rank(dst + row, (unsigned)r) = own[row];
      }
    }
    cluster_sync_all();
    // 3. w = p - (tau/2)(p.v) v and the rank-2 update
    double g = 0.0;
    for (int l = j + 1 + tid; l < n; l += PF_TRI_DS_NT) g = fma(pj[l], vb[l], g);
    g = block_sum_act(g, sh, m);
    if (tid == 0) rf[0] = 0.5 * t * g;   // once, not in every warp (FP64 pipe)
    __syncthreads();
    const double cc = rf[0];
    for (int l = j + 1 + tid; l < n; l += PF_TRI_DS_NT) wb[l] = pj[l] - cc * vb[l];
    __syncthreads();
    // over all (own column, row) pairs at once: with few rows per column a loop over the columns one
    // after another left most threads idle (one CTA at n = 64: 18 us per column)
    {
      const int kend = (int)rank < n ? min(ldc, (n - 1 - (int)rank) / (int)cs + 1) : 0;   // own columns c < n
      const int64_t tot = (int64_t)max(kend - k0, 0) * m;
      for (int64_t idx = tid; idx < tot; idx += PF_TRI_DS_NT) {
        const int k = k0 + (int)(idx / m), l = j + 1 + (int)(idx % m);
        const int c = k * (int)cs + (int)rank;
        double* a = cols + (size_t)k * n + l;
        *a = rank2_entry(*a, vb[l], wb[c], wb[l], vb[c]);
      }
    }
    if (j + 3 < n) {
      double* xn = xb + (size_t)((j + 1) & 1) * n;
      for (int l = j + 1 + tid; l < n; l += PF_TRI_DS_NT) xn[l] = rank2_entry(xn[l], vb[l], wb[j + 1], wb[l], vb[j + 1]);
    }
    __syncthreads();
  }
  for (int k = 0; k < ldc; ++k) {
    const int c = k * (int)cs + (int)rank;
    if (c < n)
      for (int r = tid; r < n; r += PF_TRI_DS_NT) Aw[(int64_t)c * n + r] = cols[(size_t)k * n + r];
  }
  cluster_sync_all();   // no CTA leaves while another may still write its shared memory
}

static size_t tridiag_dsmem_bytes(int n, int cs) {
  const int ldc = (n + cs - 1) / cs;
  return ((size_t)ldc * n + 6 * (size_t)n) * sizeof(double);
}

// Cluster size for the distributed-shared-memory tridiagonalisation of order n (0: not possible):
// the largest of 16, 8, 4, 2 whose per-CTA share of the matrix fits in shared memory and of which
// the device runs a cluster.
static int tridiag_dsmem_cluster_query(int n);
static int tridiag_dsmem_cluster(int n) {
  static std::mutex mu;
  static std::map<int, int> memo;
  std::lock_guard<std::mutex> lock(mu);
  auto it = memo.find(n);
  if (it != memo.end()) return it->second;
  return memo[n] = tridiag_dsmem_cluster_query(n);
}
static int tridiag_dsmem_cluster_query(int n) {
  static int smem_max = -1;
  if (smem_max < 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) v = 0;
    cudaGetLastError();
    smem_max = v;
  }
  auto kern = tridiag_dsmem_kernel;
  for (int c : {16, 8, 4, 2}) {
    const size_t bytes = tridiag_dsmem_bytes(n, c);
    if (bytes + 1024 > (size_t)smem_max) continue;
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (raise_smem_limit((const void*)kern, bytes) != PF_OK) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c, 1, 1);
    cfg.blockDim = dim3(PF_TRI_DS_NT, 1, 1);
    cfg.dynamicSmemBytes = bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) == cudaSuccess && ncl >= 1) return c;
    cudaGetLastError();
  }
  return 0;
}

static pf_status tridiag_dsmem(double* Aw, int n, double* d, double* e, double* tau, int cs, cudaStream_t st) {
  const size_t bytes = tridiag_dsmem_bytes(n, cs);
  PF_TRY(raise_smem_limit((const void*)tridiag_dsmem_kernel, bytes));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cs, 1, 1);
  cfg.blockDim = dim3(PF_TRI_DS_NT, 1, 1);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PF_COUNT(1);
  PF_CUDA(cudaLaunchKernelEx(&cfg, tridiag_dsmem_kernel, Aw, n, (n + cs - 1) / cs, d, e, tau));
  return PF_OK;
}

// Largest cluster (16, else 8, 4, 2) the device can run for the fused tridiagonalisation;
// 0 when clusters are unavailable.
static int tridiag_cluster_size() {
  static const int cs = [] {
    auto kern = tridiag_cluster_kernel;
    cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int c : {16, 8, 4, 2}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)c, 1, 1);
      cfg.blockDim = dim3(PF_TRI_NT, 1, 1);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)c;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters >= 1) return c;
      cudaGetLastError();
    }
    return 0;
  }();
  return cs;
}

static pf_status tridiag_cluster(double* Aw, int n, double* d, double* e, double* tau, double* p, int cs,
                                 cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cs, 1, 1);
  cfg.blockDim = dim3(PF_TRI_NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PF_COUNT(1);
  PF_CUDA(cudaLaunchKernelEx(&cfg, tridiag_cluster_kernel, Aw, n, d, e, tau, p));
  return PF_OK;
}

__global__ void tri_finish_kernel(const double* Aw, int n, double* d, double* e, double* tau) {
  if (threadIdx.x != 0) return;
  if (n == 1) {
    d[0] = Aw[0];
    return;
  }
  d[n - 2] = Aw[(int64_t)(n - 2) * n + n - 2];
  d[n - 1] = Aw[(int64_t)(n - 1) * n + n - 1];
  e[n - 2] = Aw[(int64_t)(n - 2) * n + n - 1];
  tau[n - 2] = 0.0;
}

// Sturm count: number of eigenvalues of T below x, from the pivots of the LDL^T factorisation of
// T - x I (e2[i] = e[i]^2); pivmin guards tiny pivots.
template <typename T>
__device__ int sturm_count(const T* d, const T* e2, int n, T x, T pivmin) {
  int cnt = 0;
  T q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  if (q < T(0)) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < T(0)) ++cnt;
  }
  return cnt;
}

// Pair-float a - b and a / b for the Sturm counts (stored form in, stored form out).  a - b: two_sum
// of the high parts, the low parts added to its error, renormalised.  a / b: Dekker's division, the
// FP32 quotient q1 of the high parts and the quotient of the remainder a - b q1 (formed with two_prod)
// as the low part; about 2^-44 relative.
__device__ __forceinline__ df2 dfe_sub(df2 a, df2 b) {
  const float s = __fsub_rn(a.hi, b.hi);
  const float w = __fsub_rn(s, a.hi);
  float t = __fsub_rn(__fsub_rn(a.hi, __fsub_rn(s, w)), __fadd_rn(b.hi, w));
  t = __fadd_rn(t, __fsub_rn(a.lo, b.lo));
  return df_norm(df2(s, t));
}
__device__ __forceinline__ df2 dfe_div(df2 a, df2 b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float p = __fmul_rn(b.hi, q1);
  const float e = __fmaf_rn(b.hi, q1, -p);   // b.hi q1 = p + e exactly
  float r = __fsub_rn(__fsub_rn(a.hi, p), e);
  r = __fadd_rn(r, a.lo);
  r = __fsub_rn(r, __fmul_rn(b.lo, q1));
  return df_norm(df2(q1, __fdiv_rn(r, b.hi)));
}

// The Sturm count in pair-float on the scaled matrix (d and e^2 as pairs).  |e^2 / q| stays below
// 1 / FLT_MIN because |q| >= pivmin = FLT_MIN max(1, max e^2); a non-finite pivot is taken as the
// +infinity it stands for.
__device__ int sturm_count_df(const df2* d, const df2* e2, int n, df2 x, float pivmin) {
  int cnt = 0;
  df2 q = dfe_sub(d[0], x);
  if (fabsf(q.hi) < pivmin) q = df2(-pivmin, 0.0f);
  if (q.hi < 0.0f) ++cnt;
  for (int i = 1; i < n; ++i) {
    q = dfe_sub(dfe_sub(d[i], x), dfe_div(e2[i - 1], q));
    if (!(fabsf(q.hi) <= 3.0e38f)) q = df2(3.0e38f, 0.0f);
    if (fabsf(q.hi) < pivmin) q = df2(-pivmin, 0.0f);
    if (q.hi < 0.0f) ++cnt;
  }
  return cnt;
}

// e2 = e^2 in FP64, and T scaled by sc (a power of two, so that ||T|| sc < 1) in FP32: df = d sc,
// e2f = (e sc)^2, and in pair-float: ddf = d sc, e2df = (e sc)^2.
__global__ void sturm_prep_kernel(const double* d, const double* e, int n, double sc, double* e2, float* df,
                                  float* e2f, df2* ddf, df2* e2df) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ei = i < n - 1 ? e[i] : 0.0;
  e2[i] = ei * ei;
  df[i] = (float)(d[i] * sc);
  const float ef = (float)(ei * sc);
  e2f[i] = ef * ef;
  ddf[i] = df2(d[i] * sc);
  e2df[i] = df2((ei * sc) * (ei * sc));
}

// Multisection, one warp per requested eigenvalue (index k of the ascending order): each round the
// 32 lanes take Sturm counts at 32 evenly spaced points of (lo, hi] (lane 31 at hi), and the warp
// keeps the sub-interval between the last point with fewer than k+1 eigenvalues below it and the
// first with at least k+1, a 32-fold shrink (five bisection steps) per round.
//   - The first rounds count in FP32 on the scaled matrix until the interval is below delta.  An FP32
//     count is the exact count of a matrix within ~9 eps_32 ||T|| of T (the backward error of the
//     LDL^T recurrence, with the rounding of d, e and the shift), so the FP32 interval widened by
//     delta (2^-17 ||T||, 14 times that) holds eigenvalue k of T.
//   - The FP64 rounds continue from there to the rounding level.  Their first round places its points
//     at both ends of the interval and, should the ends not bracket eigenvalue k, starts again from
//     the Gershgorin interval [gl, gu] (widened by rounding).
// One multisection round of a warp on (lo, hi] with the count routine cnt_at(x): 32 points (lane 31 at
// hi), or, with ends set, 32 points from lo to hi inclusive, and then false when the ends do not bracket
// eigenvalue k (the caller starts again from the whole interval).  Returns false also when the round
// made no progress at this resolution.
template <typename CountAt>
__device__ __forceinline__ bool multisection_round(double& lo, double& hi, bool ends, int k, int lane,
                                                   CountAt cnt_at, bool& bracket_ok) {
  const double x = lane == 31 ? hi : lo + (hi - lo) * (ends ? (double)lane / 31.0 : (double)(lane + 1) / 32.0);
  const unsigned mask = __ballot_sync(0xffffffffu, cnt_at(x) >= k + 1);
  bracket_ok = !ends || (!(mask & 1u) && (mask >> 31));
  if (!bracket_ok) return false;
  const int first = mask ? __ffs(mask) - 1 : 31;
  const double nhi = __shfl_sync(0xffffffffu, x, first);
  const double nlo = first > 0 ? __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0) : lo;
  if (nhi >= hi && nlo <= lo) return false;
  lo = nlo;
  hi = nhi;
  return true;
}

// Multisection, one warp per requested eigenvalue (index k of the ascending order): each round the
// 32 lanes take Sturm counts at 32 evenly spaced points of (lo, hi] (lane 31 at hi), and the warp
// keeps the sub-interval between the last point with fewer than k+1 eigenvalues below it and the
// first with at least k+1, a 32-fold shrink (five bisection steps) per round.  The rounds run in three
// precisions, each while the interval is wider than what the next can resolve cheaply:
//   - FP32 on the scaled matrix until the interval is below delta32 = 2^-17 ||T||.  An FP32 count is the
//     exact count of a matrix within ~9 eps_32 ||T|| of T (the backward error of the LDL^T recurrence,
//     with the rounding of d, e and the shift), so the interval widened by delta32 (14 times that)
//     holds eigenvalue k of T;
//   - pair-float (about 2^-44) on the scaled matrix until the interval is below deltadf = 2^-38 ||T||,
//     the same argument with eps = 2^-44 (a margin of ~8);
//   - FP64 to the rounding level; an FP64 division is ~1000 cycles of dependent operations, a
//     pair-float one ~100, so the FP64 rounds are kept to the last ~15 bits.
// The first round of the pair-float and FP64 stages places its points at both ends of the widened
// interval and, should they not bracket eigenvalue k, the stage starts again from the Gershgorin
// interval [gl, gu] (widened by rounding).
__global__ void bisect_kernel(const double* d, const double* e2, const float* df, const float* e2f, const df2* ddf,
                              const df2* e2df, int n, const int* idx, int q, double* w, double gl, double gu,
                              double pivmin, double sc, float pivminf, double delta32, double deltadf) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= q) return;   // uniform per warp
  const int k = idx[warp];
  float lof = __double2float_rd(gl * sc), hif = __double2float_ru(gu * sc);
  const float deltaf = (float)(delta32 * sc);
  for (int it = 0; it < 8 && hif - lof > deltaf; ++it) {
    const float x = lane == 31 ? hif : lof + (hif - lof) * ((float)(lane + 1) / 32.0f);
    const int cnt = sturm_count<float>(df, e2f, n, x, pivminf);
    const unsigned mask = __ballot_sync(0xffffffffu, cnt >= k + 1);
    const int first = mask ? __ffs(mask) - 1 : 31;
    const float nhi = __shfl_sync(0xffffffffu, x, first);
    const float nlo = first > 0 ? __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0) : lof;
    if (nhi >= hif && nlo <= lof) break;
    lof = nlo;
    hif = nhi;
  }
  double lo = fmax(gl, (double)lof / sc - delta32), hi = fmin(gu, (double)hif / sc + delta32);
  auto count_df = [&](double x) { return sturm_count_df(ddf, e2df, n, df2(x * sc), pivminf); };
  bool ends = true, ok = true;
  for (int it = 0; it < 16 && hi - lo > deltadf; ++it) {
    const bool moved = multisection_round(lo, hi, ends, k, lane, count_df, ok);
    if (!ok) {
      lo = gl;
      hi = gu;
    } else if (!moved) {
      break;
    }
    ends = false;
  }
  lo = fmax(gl, lo - deltadf);
  hi = fmin(gu, hi + deltadf);
  auto count_d = [&](double x) { return sturm_count<double>(d, e2, n, x, pivmin); };
  ends = true;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;
    const bool moved = multisection_round(lo, hi, ends, k, lane, count_d, ok);
    if (!ok) {
      lo = gl;
      hi = gu;
    } else if (!moved) {
      break;
    }
    ends = false;
  }
  if (lane == 0) w[warp] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_unit(uint64_t a) {
  uint64_t z = a + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// One CTA per cluster [cs[c], cs[c+1]) of selected eigenvalues.  Thread 0 factors
// T - lambda I (tridiagonal LU with partial pivoting, the pivots kept as reciprocals) and runs the two
// triangular solves, which are sequential recurrences (carried in registers); the whole CTA does the
// Gram-Schmidt against the cluster's earlier members and the normalisation.  The factors live in
// shared memory when smem_lu is set (6 n doubles of dynamic shared memory), else in lu.
__global__ void inviter_kernel(const double* d, const double* e, int n, const double* w, const int* cs, int ncl,
                               double* Y, double* lu, double tnorm, int smem_lu) {
  extern __shared__ __align__(16) double lus[];
  __shared__ double sh[32];
  const int c = blockIdx.x;
  if (c >= ncl) return;
  const int t = threadIdx.x;
  double* dl = smem_lu ? lus : lu + (int64_t)c * 6 * n;
  double* rd = dl + n;    // reciprocals of U's diagonal
  double* du = rd + n;
  double* du2 = du + n;
  double* b = du2 + n;
  double* piv = b + n;    // 0/1 flags stored as doubles
  const double eps = 2.2e-16;
  const double pertol = 10.0 * eps * tnorm;
  double lam_prev = -1e300;
  for (int p = cs[c]; p < cs[c + 1]; ++p) {
    double lam = w[p];
    if (p > cs[c] && lam - lam_prev < pertol) lam = lam_prev + pertol;
    lam_prev = lam;
    double* y = Y + (int64_t)p * n;
    for (int i = t; i < n; i += blockDim.x) y[i] = hash_unit(((uint64_t)p << 32) ^ (uint64_t)i);
    if (t == 0) {
      // T - lam I = P L U: U has the diagonal 1/rd, the superdiagonals du, du2; L the multipliers dl
      double di = d[0] - lam;   // running diagonal entry of row i
      double ui = n > 1 ? e[0] : 0.0;   // running first superdiagonal entry of row i
      for (int i = 0; i < n - 1; ++i) {
        const double sub = e[i];               // T(i+1, i)
        const double dn = d[i + 1] - lam;      // T(i+1, i+1)
        const double un = i < n - 2 ? e[i + 1] : 0.0;   // T(i+1, i+2)
        if (fabs(di) >= fabs(sub)) {
          const double f = di != 0.0 ? sub / di : 0.0;
          dl[i] = f;
          du[i] = ui;
          du2[i] = 0.0;
          piv[i] = 0.0;
          rd[i] = di;
          di = dn - f * ui;
          ui = un;
        } else {
          const double f = di / sub;
          dl[i] = f;
          du[i] = dn;
          du2[i] = un;
          piv[i] = 1.0;
          rd[i] = sub;
          di = ui - f * dn;
          ui = -f * un;
        }
      }
      rd[n - 1] = di;
      for (int i = 0; i < n; ++i) rd[i] = 1.0 / (rd[i] != 0.0 ? rd[i] : (pertol > 0 ? pertol : 1e-300));
    }
    __syncthreads();
    for (int it = 0; it < 4; ++it) {
      for (int i = t; i < n; i += blockDim.x) b[i] = y[i];
      __syncthreads();
      if (t == 0) {
        // L solve with the row interchanges
        double bi = b[0];
        for (int i = 0; i < n - 1; ++i) {
          const double bn = b[i + 1];
          if (piv[i] != 0.0) {
            b[i] = bn;
            bi = bi - dl[i] * bn;
          } else {
            b[i] = bi;
            bi = bn - dl[i] * bi;
          }
        }
        b[n - 1] = bi;
        // U solve
        double x1 = b[n - 1] * rd[n - 1], x2 = 0.0;
        b[n - 1] = x1;
        for (int i = n - 2; i >= 0; --i) {
          const double x = (b[i] - du[i] * x1 - du2[i] * x2) * rd[i];
          b[i] = x;
          x2 = x1;
          x1 = x;
        }
      }
      __syncthreads();
      // orthogonalise against earlier members of the cluster (twice)
      for (int pass = 0; pass < 2; ++pass)
        for (int q = cs[c]; q < p; ++q) {
          const double* z = Y + (int64_t)q * n;
          double g = 0.0;
          for (int i = t; i < n; i += blockDim.x) g = fma(z[i], b[i], g);
          g = block_sum(g, sh);
          for (int i = t; i < n; i += blockDim.x) b[i] -= g * z[i];
          __syncthreads();
        }
      double nrm = 0.0;
      for (int i = t; i < n; i += blockDim.x) nrm = fma(b[i], b[i], nrm);
      nrm = sqrt(block_sum(nrm, sh));
      if (!(nrm > 0.0)) nrm = 1.0;
      for (int i = t; i < n; i += blockDim.x) y[i] = b[i] / nrm;
      __syncthreads();
    }
  }
}

// z = H_0 H_1 ... H_{n-3} y for the column of Y given by blockIdx.x; Z column-major, ldz.
__global__ void backtransform_kernel(const double* Aw, const double* tau, int n, const double* Y, double* Z, int ldz) {
  extern __shared__ double ys[];
  __shared__ double sh[32];
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) ys[i] = Y[(int64_t)c * n + i];
  __syncthreads();
  for (int j = n - 3; j >= 0; --j) {
    const double t = tau[j];
    if (t == 0.0) continue;
    const int m = n - j - 1;
    const double* v = Aw + (int64_t)j * n + j + 1;
    double g = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) g = fma(v[i], ys[j + 1 + i], g);
    g = block_sum_act(g, sh, m);
    const double f = t * g;
    for (int i = threadIdx.x; i < m; i += blockDim.x) ys[j + 1 + i] -= f * v[i];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Z[(int64_t)c * ldz + i] = ys[i];
}

pf_status sym_eig_select(const double* A, int lda, int n, const int* idx_host, int q, double* w_host, double* Z,
                         int ldz, void* work, size_t work_bytes, cudaStream_t st) {
  if (n < 1 || q < 1 || q > n || ldz < n) return PF_EINVAL;
  EigLayout L = eig_layout(n, q);
  if (L.total > work_bytes) return PF_EINVAL;
  char* wb = (char*)work;
  double* Aw = (double*)(wb + L.aw);
  double* d = (double*)(wb + L.d);
  double* e = (double*)(wb + L.e);
  double* tau = (double*)(wb + L.tau);
  double* p = (double*)(wb + L.p);
  double* w = (double*)(wb + L.w);
  double* Y = (double*)(wb + L.y);
  double* lu = (double*)(wb + L.lu);
  int* cl = (int*)(wb + L.cl);
  int* idx_dev = cl + (q + 2);
  const int64_t nn = (int64_t)n * n;
  eig_copy_kernel<<<(unsigned)ceil_div(nn, 256), 256, 0, st>>>(A, lda, n, Aw);
  PF_LAUNCH_CHECK("eig_copy_kernel");
  // Which form, by order (measured per call, ms; the forms after the changes that gave each its
  // present shape):
  //   n      DSMEM cluster   two launches   four launches
  //   252        1.73            3.33           4.31
  //   400        3.74            5.77           7.23
  //   512        6.10            7.83           9.66
  //   616        8.92            9.65          11.98
  //   900         --            16.00          19.43
  //   1400        --            30.47          34.59
  // The DSMEM cluster kernel wherever its share of the matrix fits in shared memory (n up to ~620),
  // the L2-staged cluster kernel as its fallback for n <= 400, two launches per column up to 3000
  // (v and w of a column in 48 KB of shared memory), four above (the same bits as two).
  const int dcs = n <= 640 ? tridiag_dsmem_cluster(n) : 0;
  const int ccs = (dcs == 0 && n <= 400) ? tridiag_cluster_size() : 0;
  if (dcs > 0) {
    PF_TRY(tridiag_dsmem(Aw, n, d, e, tau, dcs, st));
  } else if (ccs > 0) {
    PF_TRY(tridiag_cluster(Aw, n, d, e, tau, p, ccs, st));
  } else if (n <= 3000) {
    unsigned* ticket = (unsigned*)(wb + L.ticket);
    PF_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), st));
    for (int j = 0; j + 2 < n; ++j) {
      const int m = n - j - 1;
      const size_t vsm = (size_t)m * sizeof(double);
      house_symv_kernel<<<(unsigned)ceil_div((int64_t)m * 32, 256), 256, vsm, st>>>(Aw, n, j, d, e, tau, p, ticket);
      rank2_vw_kernel<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)m * m, 256), 296), 256, 2 * vsm, st>>>(Aw, n, j,
                                                                                                          p);
      PF_COUNT(2);
    }
  } else {
    for (int j = 0; j + 2 < n; ++j) {
      const int m = n - j - 1;
      house_kernel<<<1, 256, 0, st>>>(Aw, n, j, d, e, tau);
      symv_kernel<<<(unsigned)ceil_div((int64_t)m * 32, 256), 256, 0, st>>>(Aw, n, j, tau, p);
      wvec_kernel<<<1, 256, 0, st>>>(Aw, n, j, tau, p);
      rank2_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(Aw, n, j, p);
      PF_COUNT(4);
    }
  }
  tri_finish_kernel<<<1, 32, 0, st>>>(Aw, n, d, e, tau);
  PF_LAUNCH_CHECK("tridiagonalisation");
  PF_CUDA(cudaMemcpyAsync(idx_dev, idx_host, q * sizeof(int), cudaMemcpyHostToDevice, st));
  std::vector<double> dh(n), eh(n);
  PF_CUDA(cudaMemcpyAsync(dh.data(), d, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  PF_CUDA(cudaMemcpyAsync(eh.data(), e, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  PF_CUDA(cudaStreamSynchronize(st));
  // Gershgorin interval of T, widened by rounding, and the pivot guard
  double gl = dh[0], gu = dh[0], maxe2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(eh[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(eh[i]) : 0.0);
    gl = std::min(gl, dh[i] - r);
    gu = std::max(gu, dh[i] + r);
    if (i < n - 1) maxe2 = std::max(maxe2, eh[i] * eh[i]);
  }
  const double tn = std::max(std::fabs(gl), std::fabs(gu));
  gl -= 2.0 * 2.2e-16 * tn * n + 1e-300;
  gu += 2.0 * 2.2e-16 * tn * n + 1e-300;
  const double pivmin = 2.3e-308 * std::max(1.0, maxe2);
  // the FP32 rounds' scale: a power of two with tn sc in [0.5, 1)
  int ex = 0;
  std::frexp(tn, &ex);
  const double sc = tn > 0.0 ? std::ldexp(1.0, -ex) : 1.0;
  const float pivminf = 1.2e-38f * (float)std::max(1.0, maxe2 * sc * sc);
  double* e2 = (double*)(wb + L.sturm);
  float* df = (float*)(e2 + n);
  float* e2f = df + n;
  df2* ddf = (df2*)(e2f + n);
  df2* e2df = ddf + n;
  sturm_prep_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(d, e, n, sc, e2, df, e2f, ddf, e2df);
  // one warp per CTA: the Sturm counts are bound by the FP64 pipe, and q warps packed eight to a
  // CTA ran on q / 8 SMs (n = 900, q = 150: 10.5 ms on 19 SMs)
  bisect_kernel<<<(unsigned)q, 32, 0, st>>>(d, e2, df, e2f, ddf, e2df, n, idx_dev, q, w, gl, gu, pivmin, sc, pivminf,
                                            std::ldexp(tn, -17), std::ldexp(tn, -38));
  PF_COUNT(1);   // sturm_prep_kernel
  PF_LAUNCH_CHECK("bisect_kernel");
  PF_CUDA(cudaMemcpyAsync(w_host, w, q * sizeof(double), cudaMemcpyDeviceToHost, st));
  PF_CUDA(cudaStreamSynchronize(st));
  double tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    double r = fabs(dh[i]) + (i > 0 ? fabs(eh[i - 1]) : 0.0) + (i < n - 1 ? fabs(eh[i]) : 0.0);
    tnorm = std::max(tnorm, r);
  }
  // clusters: consecutive requested indices whose eigenvalues are within 1e-6 ||T||.  An eigenvalue
  // separated from its neighbours by a gap g gets its vector from its own inverse iteration, accurate
  // to ~eps ||T|| / g (2e-10 at g = 1e-6 ||T||; the Ritz vectors are rotated by a Rayleigh-Ritz in H
  // afterwards); closer ones are kept orthogonal by Gram-Schmidt inside their cluster, which one CTA
  // walks sequentially.  With LAPACK's 1e-3 ||T|| the top Ritz values of the filtered H_L (spaced
  // ~3e-3 apart) chained into long clusters that serialised the whole step.
  std::vector<int> cs;
  cs.push_back(0);
  for (int i = 1; i < q; ++i) {
    bool same = idx_host[i] == idx_host[i - 1] + 1 && (w_host[i] - w_host[i - 1]) <= 1e-6 * tnorm;
    if (!same) cs.push_back(i);
  }
  cs.push_back(q);
  const int ncl = (int)cs.size() - 1;
  PF_CUDA(cudaMemcpyAsync(cl, cs.data(), cs.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  // the LU factors in shared memory up to n = 2000 (96 KB)
  const int smem_lu = n <= 2000 ? 1 : 0;
  const size_t lu_smem = smem_lu ? (size_t)6 * n * sizeof(double) : 0;
  if (lu_smem > 48 * 1024) PF_TRY(raise_smem_limit((const void*)inviter_kernel, (size_t)6 * 2000 * sizeof(double)));
  inviter_kernel<<<(unsigned)ncl, 256, lu_smem, st>>>(d, e, n, w, cl, ncl, Y, lu, tnorm, smem_lu);
  PF_LAUNCH_CHECK("inviter_kernel");
  const size_t smem = (size_t)n * sizeof(double);
  if (smem > 48 * 1024) {
    if (smem > 200 * 1024) return PF_EINVAL;
    PF_TRY(raise_smem_limit((const void*)backtransform_kernel, smem));
  }
  backtransform_kernel<<<q, 256, smem, st>>>(Aw, tau, n, Y, Z, ldz);
  PF_LAUNCH_CHECK("backtransform_kernel");
  PF_CUDA(cudaStreamSynchronize(st));   // the host cluster vectors go out of scope
  return PF_OK;
}

}  // namespace pf

using namespace pf;

pf_status pf_sym_eig_select(const double* A, int32_t lda, int32_t n, const int32_t* idx, int32_t q, double* w,
                            double* Z, int32_t ldz, pf_stream_t stream) {
  if (!A || !idx || !w || !Z || n < 1 || n > 25000 || q < 1 || q > n || lda < n || ldz < n) return PF_EINVAL;
  for (int i = 0; i < q; ++i)
    if (idx[i] < 0 || idx[i] >= n) return PF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = eig_workspace_bytes(n, q);
  void* work = dev_alloc(bytes, st);
  if (!work) return PF_ENOMEM;
  const pf_status r = sym_eig_select(A, lda, n, idx, q, w, Z, ldz, work, bytes, st);
  dev_free(work, st);
  return r;
}
