// (a5) The fused Clenshaw-SpMM step and the K-step filter application.
//
// Paper Sec. 4.4, Eq. clenshaw_chebyshev_prod: with b_{K+1} = b_{K+2} = 0,
//     b_i = a_i V + 2 H~ b_{i+1} - b_{i+2}     (i = K..1)
//     P(H~) V = a_0 V + H~ b_1 - b_2.
// One launch computes out = a V + alpha (H~ B1) - beta B2 for a whole D x s block.
//
// Layout: blocks are D x s row-major, so the s entries of a row are one contiguous
// segment of s*sizeof(T) bytes.  A row is owned by a group of G lanes, each holding
// E = s/G consecutive entries as one 16-byte vector where possible.  For every stored
// (column, value) pair of the row the group reads the neighbour row B1[col, :] as one
// coalesced segment, so each matrix entry is loaded once and reused s times.  All
// operands keep the default cache policy: every array of a step is touched again by
// the next step (V and the matrix every step, out becomes the next B1, B2's lines are
// rewritten in place), so whatever of the step's working set fits in L2 stays there.
#include "common.cuh"
#include <algorithm>

namespace pf {

template <typename T, int E> struct Vec;
template <> struct Vec<float, 1> { float x[1]; };
template <> struct Vec<float, 2> { float x[2]; };
template <> struct __align__(16) Vec<float, 4> { float x[4]; };
template <> struct Vec<double, 1> { double x[1]; };
template <> struct __align__(16) Vec<double, 2> { double x[2]; };

template <typename T, int E>
__device__ __forceinline__ Vec<T, E> ld_default(const T* p) {
  Vec<T, E> r;
  if constexpr (sizeof(T) * E == 16) {
    if constexpr (sizeof(T) == 4) {
      float4 v = __ldg(reinterpret_cast<const float4*>(p));
      r.x[0] = v.x; r.x[1] = v.y; r.x[2] = v.z; r.x[3] = v.w;
    } else {
      double2 v = __ldg(reinterpret_cast<const double2*>(p));
      r.x[0] = v.x; r.x[1] = v.y;
    }
  } else if constexpr (sizeof(T) * E == 8 && sizeof(T) == 4) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    r.x[0] = v.x; r.x[1] = v.y;
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) r.x[e] = __ldg(p + e);
  }
  return r;
}

// Coherent load for B2, which the same kernel overwrites (out may alias it).
template <typename T, int E>
__device__ __forceinline__ Vec<T, E> ld_plain(const T* p) {
  Vec<T, E> r;
  if constexpr (sizeof(T) * E == 16) {
    if constexpr (sizeof(T) == 4) {
      float4 v = *reinterpret_cast<const float4*>(p);
      r.x[0] = v.x; r.x[1] = v.y; r.x[2] = v.z; r.x[3] = v.w;
    } else {
      double2 v = *reinterpret_cast<const double2*>(p);
      r.x[0] = v.x; r.x[1] = v.y;
    }
  } else if constexpr (sizeof(T) * E == 8 && sizeof(T) == 4) {
    float2 v = *reinterpret_cast<const float2*>(p);
    r.x[0] = v.x; r.x[1] = v.y;
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) r.x[e] = p[e];
  }
  return r;
}

template <typename T, int E>
__device__ __forceinline__ void st_default(T* p, const Vec<T, E>& r) {
  if constexpr (sizeof(T) * E == 16) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(r.x[0], r.x[1], r.x[2], r.x[3]);
    } else {
      *reinterpret_cast<double2*>(p) = make_double2(r.x[0], r.x[1]);
    }
  } else if constexpr (sizeof(T) * E == 8 && sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(r.x[0], r.x[1]);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) p[e] = r.x[e];
  }
}

template <typename T, int S> struct Shape {
  static constexpr int E = (S * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : S;
  static constexpr int G = S / E;           // lanes per row
  static constexpr int ROWS_PER_WARP = 32 / G;
};

// out[row, :] = a V[row, :] + alpha * sum_j val[j] B1[col[j], :] - beta B2[row, :]
template <typename T, int S, bool SPMM, bool HAS_B2>
__global__ void __launch_bounds__(256) clenshaw_step_kernel(int64_t D, const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const T* __restrict__ val, const T* __restrict__ V,
                                                            const T* __restrict__ B1, const T* B2, T* out, T a,
                                                            T alpha, T beta) {
  using Sh = Shape<T, S>;
  constexpr int E = Sh::E, G = Sh::G;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t row = gtid / G;
  const int lane = (int)(gtid % G);
  if (row >= D) return;
  const int64_t off = row * S + lane * E;
  T acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = T(0);
  if constexpr (SPMM) {
    int64_t j = rp[row];
    const int64_t end = rp[row + 1];
    for (; j + 4 <= end; j += 4) {
      int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2), c3 = __ldg(col + j + 3);
      T h0 = __ldg(val + j), h1 = __ldg(val + j + 1), h2 = __ldg(val + j + 2), h3 = __ldg(val + j + 3);
      Vec<T, E> b0 = ld_default<T, E>(B1 + (int64_t)c0 * S + lane * E);
      Vec<T, E> b1 = ld_default<T, E>(B1 + (int64_t)c1 * S + lane * E);
      Vec<T, E> b2 = ld_default<T, E>(B1 + (int64_t)c2 * S + lane * E);
      Vec<T, E> b3 = ld_default<T, E>(B1 + (int64_t)c3 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        acc[e] = fma(h0, b0.x[e], acc[e]);
        acc[e] = fma(h1, b1.x[e], acc[e]);
        acc[e] = fma(h2, b2.x[e], acc[e]);
        acc[e] = fma(h3, b3.x[e], acc[e]);
      }
    }
    for (; j < end; ++j) {
      int c0 = __ldg(col + j);
      T h0 = __ldg(val + j);
      Vec<T, E> b0 = ld_default<T, E>(B1 + (int64_t)c0 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = fma(h0, b0.x[e], acc[e]);
    }
  }
  Vec<T, E> v = ld_default<T, E>(V + off);
  Vec<T, E> r;
  if constexpr (HAS_B2) {
    Vec<T, E> q = ld_plain<T, E>(B2 + off);
#pragma unroll
    for (int e = 0; e < E; ++e) r.x[e] = fma(alpha, acc[e], a * v.x[e] - beta * q.x[e]);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) r.x[e] = fma(alpha, acc[e], a * v.x[e]);
  }
  st_default<T, E>(out + off, r);
}

template <typename T, int S>
static pf_status launch_step_s(int64_t D, const int64_t* rp, const int32_t* col, const T* val, const T* V, const T* B1,
                               const T* B2, T* out, T a, T alpha, T beta, cudaStream_t st) {
  using Sh = Shape<T, S>;
  const int64_t threads = D * Sh::G;
  const unsigned grid = (unsigned)ceil_div(threads, 256);
  const bool spmm = alpha != T(0);
  const bool hb2 = beta != T(0);
  if (spmm && hb2)
    clenshaw_step_kernel<T, S, true, true><<<grid, 256, 0, st>>>(D, rp, col, val, V, B1, B2, out, a, alpha, beta);
  else if (spmm)
    clenshaw_step_kernel<T, S, true, false><<<grid, 256, 0, st>>>(D, rp, col, val, V, B1, B2, out, a, alpha, beta);
  else if (hb2)
    clenshaw_step_kernel<T, S, false, true><<<grid, 256, 0, st>>>(D, rp, col, val, V, B1, B2, out, a, alpha, beta);
  else
    clenshaw_step_kernel<T, S, false, false><<<grid, 256, 0, st>>>(D, rp, col, val, V, B1, B2, out, a, alpha, beta);
  PF_LAUNCH_CHECK("clenshaw_step_kernel");
  return PF_OK;
}

template <typename T>
static pf_status launch_step(int s, int64_t D, const int64_t* rp, const int32_t* col, const T* val, const T* V,
                             const T* B1, const T* B2, T* out, T a, T alpha, T beta, cudaStream_t st) {
  switch (s) {
    case 1: return launch_step_s<T, 1>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st);
    case 2: return launch_step_s<T, 2>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st);
    case 4: return launch_step_s<T, 4>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st);
    case 8: return launch_step_s<T, 8>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st);
    case 16: return launch_step_s<T, 16>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st);
    case 32: return launch_step_s<T, 32>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st);
    case 64: return launch_step_s<T, 64>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st);
  }
  return PF_EINVAL;
}

static bool valid_s(int s) { return s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32 || s == 64; }

pf_status clenshaw_step_raw(int64_t D, const int64_t* row_ptr, const int32_t* col, const void* val, int prec, int s,
                            const void* V, const void* B1, const void* B2, void* out, double a, double alpha,
                            double beta, cudaStream_t st) {
  if (!valid_s(s) || D <= 0 || !V || !out) return PF_EINVAL;
  if (alpha != 0.0 && (!B1 || !val)) return PF_EINVAL;
  if (beta != 0.0 && !B2) return PF_EINVAL;
  if (beta != 0.0 && beta != 1.0) return PF_EINVAL;
  if (prec == PF_F64)
    return launch_step<double>(s, D, row_ptr, col, (const double*)val, (const double*)V, (const double*)B1,
                               (const double*)B2, (double*)out, a, alpha, beta, st);
  if (prec == PF_F32)
    return launch_step<float>(s, D, row_ptr, col, (const float*)val, (const float*)V, (const float*)B1,
                              (const float*)B2, (float*)out, (float)a, (float)alpha, (float)beta, st);
  return PF_EINVAL;
}

// K-step recurrence.  b_i lives in aux[i & 1]: step i reads b_{i+1} = aux[(i+1)&1] and
// overwrites b_{i+2} (= aux[i&1]) with b_i.
pf_status filter_apply_raw(const Ham* H, int prec, int s, const void* V, void* W, const double* coeffs, const void*,
                           int K, void* aux0, void* aux1, cudaStream_t st) {
  if (K < 1 || !coeffs) return PF_EINVAL;
  const void* val = prec == PF_F64 ? (const void*)H->val_t : (const void*)H->val32;
  void* aux[2] = {aux0, aux1};
  // i = K: b_K = a_K V
  PF_TRY(clenshaw_step_raw(H->D, H->row_ptr, H->col, val, prec, s, V, nullptr, nullptr, aux[K & 1], coeffs[K], 0.0,
                           0.0, st));
  for (int i = K - 1; i >= 1; --i) {
    const double beta = (i == K - 1) ? 0.0 : 1.0;
    PF_TRY(clenshaw_step_raw(H->D, H->row_ptr, H->col, val, prec, s, V, aux[(i + 1) & 1], aux[i & 1], aux[i & 1],
                             coeffs[i], 2.0, beta, st));
  }
  // P V = a_0 V + H~ b_1 - b_2
  const double beta = (K >= 2) ? 1.0 : 0.0;
  PF_TRY(clenshaw_step_raw(H->D, H->row_ptr, H->col, val, prec, s, V, aux[1], aux[0], W, coeffs[0], 1.0, beta, st));
  return PF_OK;
}

// ------------------------------------------------------------------ batched sweep
// Several filter applications W_j = P_j(H~_j) V_j (different matrices, sizes, degrees) advance
// together: launch t of a sweep performs one Clenshaw step of every item at once, over the
// concatenation of the items' rows.  Item j (degree K_j) joins at t0_j = T - (K_j + 1) so that
// all items finish at the last launch; at sweep step t it runs recurrence index
// i = K_j - (t - t0_j) with the same operands as filter_apply_raw.
struct BatchItemDev {
  int64_t D, row0;
  const int64_t* rp;
  const int32_t* col;
  const void* val;
  const void* V;
  void* W;
  void* aux0;
  void* aux1;
  const double* coeffs;
  int K, t0;
};

template <typename T, int S>
__global__ void __launch_bounds__(256) clenshaw_batch_kernel(const BatchItemDev* __restrict__ items, int n, int t,
                                                             int64_t total_rows) {
  using Sh = Shape<T, S>;
  constexpr int E = Sh::E, G = Sh::G;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t grow = gtid / G;
  const int lane = (int)(gtid % G);
  if (grow >= total_rows) return;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].row0 <= grow) lo = mid;
    else hi = mid - 1;
  }
  const BatchItemDev& it = items[lo];
  if (t < it.t0) return;
  const int K = it.K;
  const int i = K - (t - it.t0);
  const int64_t row = grow - it.row0;
  T* aux[2] = {(T*)it.aux0, (T*)it.aux1};
  const T* B1 = nullptr;
  const T* B2 = nullptr;
  T* out;
  T alpha, beta;
  if (i == K) {
    alpha = T(0); beta = T(0); out = aux[i & 1];
  } else if (i >= 1) {
    alpha = T(2); beta = (i == K - 1) ? T(0) : T(1);
    B1 = aux[(i + 1) & 1]; B2 = aux[i & 1]; out = aux[i & 1];
  } else {
    alpha = T(1); beta = (K >= 2) ? T(1) : T(0);
    B1 = aux[1]; B2 = aux[0]; out = (T*)it.W;
  }
  const T a = (T)it.coeffs[i];
  const T* __restrict__ V = (const T*)it.V;
  const T* __restrict__ val = (const T*)it.val;
  const int32_t* __restrict__ col = it.col;
  const int64_t off = row * S + lane * E;
  T acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = T(0);
  if (alpha != T(0)) {
    int64_t j = it.rp[row];
    const int64_t end = it.rp[row + 1];
    for (; j + 4 <= end; j += 4) {
      int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2), c3 = __ldg(col + j + 3);
      T h0 = __ldg(val + j), h1 = __ldg(val + j + 1), h2 = __ldg(val + j + 2), h3 = __ldg(val + j + 3);
      Vec<T, E> b0 = ld_default<T, E>(B1 + (int64_t)c0 * S + lane * E);
      Vec<T, E> b1 = ld_default<T, E>(B1 + (int64_t)c1 * S + lane * E);
      Vec<T, E> b2 = ld_default<T, E>(B1 + (int64_t)c2 * S + lane * E);
      Vec<T, E> b3 = ld_default<T, E>(B1 + (int64_t)c3 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        acc[e] = fma(h0, b0.x[e], acc[e]);
        acc[e] = fma(h1, b1.x[e], acc[e]);
        acc[e] = fma(h2, b2.x[e], acc[e]);
        acc[e] = fma(h3, b3.x[e], acc[e]);
      }
    }
    for (; j < end; ++j) {
      int c0 = __ldg(col + j);
      T h0 = __ldg(val + j);
      Vec<T, E> b0 = ld_default<T, E>(B1 + (int64_t)c0 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = fma(h0, b0.x[e], acc[e]);
    }
  }
  Vec<T, E> v = ld_default<T, E>(V + off);
  Vec<T, E> r;
  if (beta != T(0)) {
    Vec<T, E> q = ld_plain<T, E>(B2 + off);
#pragma unroll
    for (int e = 0; e < E; ++e) r.x[e] = fma(alpha, acc[e], a * v.x[e] - beta * q.x[e]);
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) r.x[e] = fma(alpha, acc[e], a * v.x[e]);
  }
  st_default<T, E>(out + off, r);
}

template <typename T, int S>
static pf_status launch_batch_s(const BatchItemDev* items, int n, int T_steps, int64_t total_rows, cudaStream_t st) {
  using Sh = Shape<T, S>;
  const unsigned grid = (unsigned)ceil_div(total_rows * Sh::G, 256);
  for (int t = 0; t < T_steps; ++t) {
    clenshaw_batch_kernel<T, S><<<grid, 256, 0, st>>>(items, n, t, total_rows);
    PF_LAUNCH_CHECK("clenshaw_batch_kernel");
  }
  return PF_OK;
}

pf_status filter_sweep(const std::vector<FilterItem>& items, void* table_dev, size_t table_bytes, void* table_host,
                       cudaStream_t st) {
  const int n = (int)items.size();
  if (n == 0) return PF_OK;
  if ((size_t)n * sizeof(BatchItemDev) > table_bytes) return PF_EINVAL;
  const int prec = items[0].prec, s = items[0].s;
  int T = 0;
  for (const auto& it : items) {
    if (it.prec != prec || it.s != s || it.K < 1) return PF_EINVAL;
    T = std::max(T, it.K + 1);
  }
  BatchItemDev* tab = static_cast<BatchItemDev*>(table_host);
  int64_t row0 = 0;
  for (int j = 0; j < n; ++j) {
    const FilterItem& it = items[j];
    BatchItemDev& b = tab[j];
    b.D = it.H->D;
    b.row0 = row0;
    b.rp = it.H->row_ptr;
    b.col = it.H->col;
    b.val = prec == PF_F64 ? (const void*)it.H->val_t : (const void*)it.H->val32;
    b.V = it.V;
    b.W = it.W;
    b.aux0 = it.aux0;
    b.aux1 = it.aux1;
    b.coeffs = it.coeffs_dev;
    b.K = it.K;
    b.t0 = T - (it.K + 1);
    row0 += it.H->D;
  }
  PF_CUDA(cudaMemcpyAsync(table_dev, tab, n * sizeof(BatchItemDev), cudaMemcpyHostToDevice, st));
  const BatchItemDev* d = static_cast<const BatchItemDev*>(table_dev);
  if (prec == PF_F64) {
    switch (s) {
      case 1: return launch_batch_s<double, 1>(d, n, T, row0, st);
      case 2: return launch_batch_s<double, 2>(d, n, T, row0, st);
      case 4: return launch_batch_s<double, 4>(d, n, T, row0, st);
      case 8: return launch_batch_s<double, 8>(d, n, T, row0, st);
      case 16: return launch_batch_s<double, 16>(d, n, T, row0, st);
      case 32: return launch_batch_s<double, 32>(d, n, T, row0, st);
      case 64: return launch_batch_s<double, 64>(d, n, T, row0, st);
    }
  } else {
    switch (s) {
      case 1: return launch_batch_s<float, 1>(d, n, T, row0, st);
      case 2: return launch_batch_s<float, 2>(d, n, T, row0, st);
      case 4: return launch_batch_s<float, 4>(d, n, T, row0, st);
      case 8: return launch_batch_s<float, 8>(d, n, T, row0, st);
      case 16: return launch_batch_s<float, 16>(d, n, T, row0, st);
      case 32: return launch_batch_s<float, 32>(d, n, T, row0, st);
      case 64: return launch_batch_s<float, 64>(d, n, T, row0, st);
    }
  }
  return PF_EINVAL;
}

size_t filter_sweep_table_bytes(int n) { return (size_t)n * sizeof(BatchItemDev); }

}  // namespace pf

using namespace pf;

extern "C" {

pf_status pf_clenshaw_step(const pf_ham* hh, int32_t prec, int32_t s, const void* V, const void* B1, const void* B2,
                           void* out, double a, double alpha, double beta, int32_t use_H, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H) return PF_EINVAL;
  const void* val;
  if (use_H) {
    if (prec != PF_F64) return PF_EINVAL;
    val = H->val;
  } else {
    if (!H->has_rescale) return PF_ESTATE;
    val = prec == PF_F64 ? (const void*)H->val_t : (const void*)H->val32;
  }
  return clenshaw_step_raw(H->D, H->row_ptr, H->col, val, prec, s, V, B1, B2, out, a, alpha, beta,
                           (cudaStream_t)stream);
}

pf_status pf_filter_apply(const pf_ham* hh, int32_t prec, int32_t s, const void* V, void* W, const double* coeffs,
                          int32_t K, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H || !V || !W || !coeffs || K < 1) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  if (prec != PF_F64 && prec != PF_F32) return PF_EINVAL;
  if (!valid_s(s)) return PF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t w = prec == PF_F64 ? 8 : 4;
  DevBuf a0, a1;
  PF_TRY(a0.alloc(H->D * s * w, st));
  PF_TRY(a1.alloc(H->D * s * w, st));
  return filter_apply_raw(H, prec, s, V, W, coeffs, nullptr, K, a0.p, a1.p, st);
}

pf_status pf_filter_apply_batch(const pf_filter_item* items, int32_t n, int32_t prec, int32_t s,
                                pf_stream_t stream) {
  if (n < 0 || (n > 0 && !items)) return PF_EINVAL;
  if (prec != PF_F64 && prec != PF_F32) return PF_EINVAL;
  if (!valid_s(s)) return PF_EINVAL;
  if (n == 0) return PF_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t w = prec == PF_F64 ? 8 : 4;
  // one device blob: per item its K+1 coefficients and two auxiliary blocks (256-B aligned)
  std::vector<size_t> coff(n), aoff(n);
  size_t total = 0;
  for (int j = 0; j < n; ++j) {
    const Ham* H = reinterpret_cast<const Ham*>(items[j].H);
    if (!H || !items[j].V || !items[j].W || !items[j].coeffs || items[j].K < 1) return PF_EINVAL;
    if (!H->has_rescale) return PF_ESTATE;
    coff[j] = total;
    total += ((size_t)(items[j].K + 1) * 8 + 255) & ~(size_t)255;
    aoff[j] = total;
    total += 2 * (((size_t)H->D * s * w + 255) & ~(size_t)255);
  }
  DevBuf blob, table;
  PF_TRY(blob.alloc(total, st));
  PF_TRY(table.alloc(filter_sweep_table_bytes(n), st));
  std::vector<double> ch;
  std::vector<FilterItem> v(n);
  for (int j = 0; j < n; ++j) {
    const Ham* H = reinterpret_cast<const Ham*>(items[j].H);
    unsigned char* base = blob.as<unsigned char>();
    PF_CUDA(cudaMemcpyAsync(base + coff[j], items[j].coeffs, (size_t)(items[j].K + 1) * 8, cudaMemcpyHostToDevice,
                            st));
    FilterItem& it = v[j];
    it.H = H;
    it.prec = prec;
    it.s = s;
    it.V = items[j].V;
    it.W = items[j].W;
    it.coeffs_host = items[j].coeffs;
    it.coeffs_dev = reinterpret_cast<const double*>(base + coff[j]);
    it.K = items[j].K;
    it.aux0 = base + aoff[j];
    it.aux1 = base + aoff[j] + (((size_t)H->D * s * w + 255) & ~(size_t)255);
  }
  std::vector<unsigned char> th(filter_sweep_table_bytes(n));
  return filter_sweep(v, table.p, table.bytes, th.data(), st);
}

}  // extern "C"
