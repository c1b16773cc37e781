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
#include "pairfloat.cuh"
#include <algorithm>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

// Pair-float entries per lane and the step kernel's resident CTAs per SM (64 registers).
#ifndef PF_DF_E
#define PF_DF_E 4
#endif
#ifndef PF_DF_MINB
#define PF_DF_MINB 4
#endif

namespace pf {

template <typename T> constexpr bool is_df = std::is_same_v<T, df2>;
// x * y + z in the step's arithmetic (one rounding for FP32 / FP64)
template <typename T> __device__ __forceinline__ T fmadd(T x, T y, T z) {
  if constexpr (is_df<T>) return df_fma(x, y, z);
  else return ::fma(x, y, z);
}
template <typename T> __device__ __forceinline__ T stored(T x) {
  if constexpr (is_df<T>) return df_norm(x);
  else return x;
}
// Coefficient i of a device table: FP64 values, or for pair-float steps pairs (hi, lo) written
// by the host (df2(double)), so that no step kernel executes an FP64 instruction.
template <typename T> __device__ __forceinline__ T load_coeff(const double* c) {
  if constexpr (is_df<T>) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(c));
    return df2(v.x, v.y);
  } else {
    return (T)__ldg(c);
  }
}
// Host: the device coefficient table of a precision (pairs for PF_DF64, else the values).
void coeff_table_host(int prec, const double* c, int n, double* out) {
  for (int i = 0; i < n; ++i) {
    if (prec == PF_DF64) {
      const df2 d(c[i]);
      memcpy(out + i, &d, 8);
    } else {
      out[i] = c[i];
    }
  }
}
static double coeff_value_host(int prec, double stored_bits) {
  if (prec != PF_DF64) return stored_bits;
  df2 d;
  memcpy(&d, &stored_bits, 8);
  return (double)d.hi + (double)d.lo;
}

template <typename T, int E> struct Vec;
template <> struct Vec<float, 1> { float x[1]; };
template <> struct Vec<float, 2> { float x[2]; };
template <> struct __align__(16) Vec<float, 4> { float x[4]; };
template <> struct Vec<double, 1> { double x[1]; };
template <> struct __align__(16) Vec<double, 2> { double x[2]; };
template <> struct Vec<df2, 1> { df2 x[1]; };
template <> struct __align__(16) Vec<df2, 2> { df2 x[2]; };
template <> struct __align__(16) Vec<df2, 4> { df2 x[4]; };
template <> struct __align__(16) Vec<df2, 8> { df2 x[8]; };

// Pair-float segment loads and stores: 16-byte vectors (one 8-byte vector for E = 1).
// MODE 0: read-only path (ld.global.nc), 1: coherent (ld.global), 2: L2 only (ld.global.cg).
template <int MODE, int E>
__device__ __forceinline__ Vec<df2, E> ld_df(const df2* p) {
  Vec<df2, E> r;
  if constexpr (E == 1) {
    const float2* q = reinterpret_cast<const float2*>(p);
    const float2 v = MODE == 0 ? __ldg(q) : MODE == 1 ? *q : __ldcg(q);
    r.x[0] = df2(v.x, v.y);
  } else {
#pragma unroll
    for (int k = 0; k < E; k += 2) {
      const float4* q = reinterpret_cast<const float4*>(p + k);
      const float4 v = MODE == 0 ? __ldg(q) : MODE == 1 ? *q : __ldcg(q);
      r.x[k] = df2(v.x, v.y);
      r.x[k + 1] = df2(v.z, v.w);
    }
  }
  return r;
}
template <int E>
__device__ __forceinline__ void st_df(df2* p, const Vec<df2, E>& r) {
  if constexpr (E == 1) {
    *reinterpret_cast<float2*>(p) = make_float2(r.x[0].hi, r.x[0].lo);
  } else {
#pragma unroll
    for (int k = 0; k < E; k += 2)
      *reinterpret_cast<float4*>(p + k) = make_float4(r.x[k].hi, r.x[k].lo, r.x[k + 1].hi, r.x[k + 1].lo);
  }
}

template <typename T, int E>
__device__ __forceinline__ Vec<T, E> ld_default(const T* p) {
  if constexpr (is_df<T>) {
    return ld_df<0, E>(p);
  } else {
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
}

// Coherent load for B2, which the same kernel overwrites (out may alias it).
template <typename T, int E>
__device__ __forceinline__ Vec<T, E> ld_plain(const T* p) {
  if constexpr (is_df<T>) {
    return ld_df<1, E>(p);
  } else {
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
}

template <typename T, int E>
__device__ __forceinline__ void st_default(T* p, const Vec<T, E>& r) {
  if constexpr (is_df<T>) {
    st_df<E>(p, r);
  } else if constexpr (sizeof(T) * E == 16) {
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

// Lanes per row.  FP32: E = 4 entries (one 16-byte vector) per lane, so an s = 32 row is 8
// lanes.  FP64: one row per warp where s allows it (E = max(1, s/32)): the FP64 step is bound
// by the FP64 pipe, and a warp that holds one row never idles lanes on a shorter neighbour
// row (about 8% faster than two rows of 16 lanes at s = 32).
// Pair-float: E = 4 pairs (two 16-byte vectors) per lane, 8 lanes per s = 32 row as in FP32:
// its step is bound by the neighbour gathers, not by arithmetic (12 FP32 operations per
// product, against one FP64 FMA at 1/64 of the FP32 rate).  Measured at XXZ L = 20, s = 32:
// 73.5 us with E = 4 against 93.3 us with E = 2 and 95.7 us with E = 8 (same bits).
template <typename T, int S> struct Shape {
  static constexpr int E = is_df<T> ? (S >= PF_DF_E ? PF_DF_E : S)
                         : sizeof(T) == 8 ? (S >= 64 ? S / 32 : 1) : ((S * (int)sizeof(T) >= 16) ? 16 / (int)sizeof(T) : S);
  static constexpr int G = S / E;           // lanes per row
  static constexpr int ROWS_PER_WARP = G >= 32 ? 1 : 32 / G;
};

// L2-only loads (ld.global.cg) for blocks the same launch rewrites between its steps.
template <typename T, int E>
__device__ __forceinline__ Vec<T, E> ld_l2(const T* p) {
  if constexpr (is_df<T>) {
    return ld_df<2, E>(p);
  } else {
    Vec<T, E> r;
    if constexpr (sizeof(T) * E == 16) {
      if constexpr (sizeof(T) == 4) {
        float4 v = __ldcg(reinterpret_cast<const float4*>(p));
        r.x[0] = v.x; r.x[1] = v.y; r.x[2] = v.z; r.x[3] = v.w;
      } else {
        double2 v = __ldcg(reinterpret_cast<const double2*>(p));
        r.x[0] = v.x; r.x[1] = v.y;
      }
    } else if constexpr (sizeof(T) * E == 8 && sizeof(T) == 4) {
      float2 v = __ldcg(reinterpret_cast<const float2*>(p));
      r.x[0] = v.x; r.x[1] = v.y;
    } else {
#pragma unroll
      for (int e = 0; e < E; ++e) r.x[e] = __ldcg(p + e);
    }
    return r;
  }
}

// A matrix value (read-only path).
template <typename T> __device__ __forceinline__ T ld_val(const T* p) {
  if constexpr (is_df<T>) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df2(v.x, v.y);
  } else {
    return __ldg(p);
  }
}

// The end of a row segment: out = fma(alpha, acc, fma(a, v, -beta q)), or fma(alpha, acc, a v)
// without the B2 term.  beta is 0 or 1; with the B2 term known present it is 1, so -beta q is -q
// (the same bits as the run-time form, where 1 * q is exact).  acol, when not null, holds one
// coefficient per column of the block (the s values of this step), used in place of a: entry e
// of the lane's segment takes acol[c0 + e], c0 the segment's first column.
template <typename T, int E, bool L2ONLY, int B2M>
__device__ __forceinline__ void row_epilogue(int64_t off, const T (&acc)[E], bool hb2, const T* __restrict__ V,
                                             const T* B2, T* out, T a, T alpha, T beta, const T* acol = nullptr,
                                             int c0 = 0) {
  Vec<T, E> v = ld_default<T, E>(V + off);
  T av[E];
#pragma unroll
  for (int e = 0; e < E; ++e) av[e] = a;
  if (acol) {
#pragma unroll
    for (int e = 0; e < E; ++e) av[e] = ld_val(acol + c0 + e);
  }
  Vec<T, E> r;
  if (hb2) {
    Vec<T, E> q;
    if constexpr (L2ONLY) q = ld_l2<T, E>(B2 + off);
    else q = ld_plain<T, E>(B2 + off);
#pragma unroll
    for (int e = 0; e < E; ++e)
      r.x[e] = stored(fmadd(alpha, acc[e], fmadd(av[e], v.x[e], B2M > 0 ? -q.x[e] : -(beta * q.x[e]))));
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) r.x[e] = stored(fmadd(alpha, acc[e], av[e] * v.x[e]));
  }
  st_default<T, E>(out + off, r);
}

// One row segment (lane's E entries) of one step:
//     out[row, :] = a V[row, :] + alpha * sum_j val[j] B1[col[j], :] - beta B2[row, :]
// SP / B2M: 1 = the SpMM / the B2 term is present, 0 = absent, -1 = decided at run time by
// alpha != 0 / beta != 0.  Every kernel of this file computes a row through this function, so
// all execution forms produce the same bits: the SpMM accumulates in column order, four
// entries per round, and the epilogue is fma(alpha, acc, fma(a, v, -beta q)) (or
// fma(alpha, acc, a v) without B2).  L2ONLY selects ld.global.cg for B1 and B2.
// VS selects the value source: 0 = the CSR value array; 1 = constant off-diagonal (the XXZ
// chain's J/(2 dE)): g for every column but the row's own, whose value is diag[row]; 2 = the
// quantum sun (row = state): diag[row] on the diagonal, the dot block's element when only dot bits
// differ, else the coupling of ray j, j the one outer bit that differs.  The structured values are
// those the CSR stores, so the bits agree with the CSR step.
template <typename T> struct ValSrc {
  const T* diag = nullptr;   // per-row diagonal of H~
  T g = T(0);                // VS 1: the one off-diagonal value
  const T* tab = nullptr;    // VS 2: the dot block of H~, 2^N x 2^N row-major
  const T* coef = nullptr;   // VS 2: the ray couplings of H~, [L]
  int L = 0, N = 0;          // VS 2: outer spins (bits 0..L-1) and dot spins (the bits above)
};
template <typename T, int S, bool L2ONLY, int SP, int B2M, int VS>
__device__ __forceinline__ void clenshaw_row_vs(int64_t row, int lane, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, const T* __restrict__ val,
                                                const T* __restrict__ V, const T* B1, const T* B2, T* out, T a,
                                                T alpha, T beta, const ValSrc<T>& vsrc, const T* acol = nullptr) {
  using Sh = Shape<T, S>;
  constexpr int E = Sh::E;
  const int64_t off = row * S + lane * E;
  T acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = T(0);
  const bool spmm = SP < 0 ? (alpha != T(0)) : (SP > 0);
  const bool hb2 = B2M < 0 ? (beta != T(0)) : (B2M > 0);
  auto ldb = [](const T* p) {
    if constexpr (L2ONLY) return ld_l2<T, E>(p);
    else return ld_default<T, E>(p);
  };
  if (spmm) {
    int64_t j = rp[row];
    const int64_t end = rp[row + 1];
    T dr = vsrc.g;
    if constexpr (VS >= 1) dr = ld_val(vsrc.diag + row);
    auto hv = [&](int64_t jj, int c) -> T {
      if constexpr (VS == 1) {
        return (int64_t)c == row ? dr : vsrc.g;
      } else if constexpr (VS == 2) {
        const uint32_t r = (uint32_t)row, x = r ^ (uint32_t)c;
        const uint32_t om = (1u << vsrc.L) - 1u;
        if (x == 0) return dr;
        if ((x & om) == 0) return ld_val(vsrc.tab + (((r >> vsrc.L) << vsrc.N) + ((uint32_t)c >> vsrc.L)));
        return ld_val(vsrc.coef + (__ffs(x & om) - 1));
      } else {
        return ld_val(val + jj);
      }
    };
    for (; j + 4 <= end; j += 4) {
      int c0 = __ldg(col + j), c1 = __ldg(col + j + 1), c2 = __ldg(col + j + 2), c3 = __ldg(col + j + 3);
      T h0 = hv(j, c0), h1 = hv(j + 1, c1), h2 = hv(j + 2, c2), h3 = hv(j + 3, c3);
      Vec<T, E> b0 = ldb(B1 + (int64_t)c0 * S + lane * E);
      Vec<T, E> b1 = ldb(B1 + (int64_t)c1 * S + lane * E);
      Vec<T, E> b2 = ldb(B1 + (int64_t)c2 * S + lane * E);
      Vec<T, E> b3 = ldb(B1 + (int64_t)c3 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        acc[e] = fmadd(h0, b0.x[e], acc[e]);
        acc[e] = fmadd(h1, b1.x[e], acc[e]);
        acc[e] = fmadd(h2, b2.x[e], acc[e]);
        acc[e] = fmadd(h3, b3.x[e], acc[e]);
      }
    }
    for (; j < end; ++j) {
      int c0 = __ldg(col + j);
      T h0 = hv(j, c0);
      Vec<T, E> b0 = ldb(B1 + (int64_t)c0 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = fmadd(h0, b0.x[e], acc[e]);
    }
  }
  row_epilogue<T, E, L2ONLY, B2M>(off, acc, hb2, V, B2, out, a, alpha, beta, acol, lane * E);
}

template <typename T, int S, bool L2ONLY, int SP, int B2M>
__device__ __forceinline__ void clenshaw_row(int64_t row, int lane, const int64_t* __restrict__ rp,
                                             const int32_t* __restrict__ col, const T* __restrict__ val,
                                             const T* __restrict__ V, const T* B1, const T* B2, T* out, T a,
                                             T alpha, T beta) {
  clenshaw_row_vs<T, S, L2ONLY, SP, B2M, 0>(row, lane, rp, col, val, V, B1, B2, out, a, alpha, beta, ValSrc<T>());
}

// One Clenshaw step over a D x s block.  rows_per_cta = 0: thread group g owns row g (one
// row per G lanes).  rows_per_cta < 0: the grid (one wave, SMs x resident CTAs) strides over
// groups of 256/G rows (the sweep order of shape_for).
template <typename T> constexpr int step_min_blocks() {
  return is_df<T> ? PF_DF_MINB : sizeof(T) == 8 ? 8 : 6;
}
template <typename T, int S, int SP, int B2M>
__global__ void __launch_bounds__(256, step_min_blocks<T>()) clenshaw_step_kernel(int64_t D, const int64_t* __restrict__ rp,
                                                            const int32_t* __restrict__ col,
                                                            const T* __restrict__ val, const T* __restrict__ V,
                                                            const T* __restrict__ B1, const T* B2, T* out, T a,
                                                            T alpha, T beta, int64_t rows_per_cta,
                                                            const T* __restrict__ acol) {
  using Sh = Shape<T, S>;
  constexpr int G = Sh::G;
  const int lane = (int)(threadIdx.x % G);
  const ValSrc<T> vs0;
  if (rows_per_cta < 0) {   // grid-stride over row groups (sweep order, or a capped grid)
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G; row < D; row += groups)
      clenshaw_row_vs<T, S, false, SP, B2M, 0>(row, lane, rp, col, val, V, B1, B2, out, a, alpha, beta, vs0, acol);
  } else {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    if (row < D)
      clenshaw_row_vs<T, S, false, SP, B2M, 0>(row, lane, rp, col, val, V, B1, B2, out, a, alpha, beta, vs0, acol);
  }
}

// Structured mapping of QREM (Eq. qrem; the custom GPU mapping of Sec. 5.8): row r of H~ holds
// d_r = diag[r] at column r and the one value g = -Gamma / dE at the L columns r ^ (1 << i).  The
// columns are generated in registers in ascending order, as the CSR stores them: r - 2^i for the
// set bits i from the highest down, then r, then r + 2^i for the unset bits from the lowest up.
// The FMA sequence (rounds of four, then the rest, in that order) is clenshaw_row's, so the
// structured and the CSR mappings give the same bits.
template <typename T, int S, int SP, int B2M>
__device__ __forceinline__ void qrem_row(int64_t row, int lane, int L, const T* __restrict__ diag, T g,
                                         const T* __restrict__ V, const T* B1, const T* B2, T* out, T a, T alpha,
                                         T beta, const T* acol) {
  using Sh = Shape<T, S>;
  constexpr int E = Sh::E;
  const int64_t off = row * S + lane * E;
  T acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = T(0);
  const bool spmm = SP < 0 ? (alpha != T(0)) : (SP > 0);
  const bool hb2 = B2M < 0 ? (beta != T(0)) : (B2M > 0);
  if (spmm) {
    const uint32_t r = (uint32_t)row;
    const uint32_t full = L >= 32 ? 0xffffffffu : ((1u << L) - 1u);
    uint32_t sb = r & full;     // set bits still to visit, highest first
    uint32_t ub = ~r & full;    // unset bits still to visit, lowest first
    bool dpend = true;
    const T dr = ld_val(diag + row);
    auto next = [&](uint32_t& c, T& h) {
      if (sb) {
        const int i = 31 - __clz(sb);
        sb ^= 1u << i;
        c = r ^ (1u << i);
        h = g;
      } else if (dpend) {
        dpend = false;
        c = r;
        h = dr;
      } else {
        const int i = __ffs(ub) - 1;
        ub &= ub - 1u;
        c = r | (1u << i);
        h = g;
      }
    };
    const int n = L + 1;
    int j = 0;
    for (; j + 4 <= n; j += 4) {
      uint32_t c0, c1, c2, c3;
      T h0, h1, h2, h3;
      next(c0, h0);
      next(c1, h1);
      next(c2, h2);
      next(c3, h3);
      Vec<T, E> b0 = ld_default<T, E>(B1 + (int64_t)c0 * S + lane * E);
      Vec<T, E> b1 = ld_default<T, E>(B1 + (int64_t)c1 * S + lane * E);
      Vec<T, E> b2 = ld_default<T, E>(B1 + (int64_t)c2 * S + lane * E);
      Vec<T, E> b3 = ld_default<T, E>(B1 + (int64_t)c3 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        acc[e] = fmadd(h0, b0.x[e], acc[e]);
        acc[e] = fmadd(h1, b1.x[e], acc[e]);
        acc[e] = fmadd(h2, b2.x[e], acc[e]);
        acc[e] = fmadd(h3, b3.x[e], acc[e]);
      }
    }
    for (; j < n; ++j) {
      uint32_t c0;
      T h0;
      next(c0, h0);
      Vec<T, E> b0 = ld_default<T, E>(B1 + (int64_t)c0 * S + lane * E);
#pragma unroll
      for (int e = 0; e < E; ++e) acc[e] = fmadd(h0, b0.x[e], acc[e]);
    }
  }
  row_epilogue<T, E, false, B2M>(off, acc, hb2, V, B2, out, a, alpha, beta, acol, lane * E);
}

template <typename T, int S, int SP, int B2M>
__global__ void __launch_bounds__(256, step_min_blocks<T>()) qrem_step_kernel(int64_t D, int L,
                                                                              const T* __restrict__ diag, T g,
                                                                              const T* __restrict__ V,
                                                                              const T* __restrict__ B1, const T* B2,
                                                                              T* out, T a, T alpha, T beta,
                                                                              int64_t rows_per_cta,
                                                                              const T* __restrict__ acol) {
  using Sh = Shape<T, S>;
  constexpr int G = Sh::G;
  const int lane = (int)(threadIdx.x % G);
  if (rows_per_cta < 0) {
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G; row < D; row += groups)
      qrem_row<T, S, SP, B2M>(row, lane, L, diag, g, V, B1, B2, out, a, alpha, beta, acol);
  } else {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    if (row < D) qrem_row<T, S, SP, B2M>(row, lane, L, diag, g, V, B1, B2, out, a, alpha, beta, acol);
  }
}

// Structured mappings that keep the CSR's columns but not its value array (clenshaw_row_vs): VS = 1,
// the XXZ chain (constant off-diagonal, per-row diagonal); VS = 2, the quantum sun (diagonal, dot
// block, ray couplings).  Same bits as the CSR step.
template <typename T, int S, int SP, int B2M, int VS>
__global__ void __launch_bounds__(256, step_min_blocks<T>()) cstruct_step_kernel(int64_t D, const int64_t* __restrict__ rp,
                                                                                 const int32_t* __restrict__ col,
                                                                                 ValSrc<T> vsrc, const T* __restrict__ V,
                                                                                 const T* __restrict__ B1, const T* B2,
                                                                                 T* out, T a, T alpha, T beta,
                                                                                 int64_t rows_per_cta,
                                                                                 const T* __restrict__ acol) {
  using Sh = Shape<T, S>;
  constexpr int G = Sh::G;
  const int lane = (int)(threadIdx.x % G);
  if (rows_per_cta < 0) {
    const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
    for (int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G; row < D; row += groups)
      clenshaw_row_vs<T, S, false, SP, B2M, VS>(row, lane, rp, col, nullptr, V, B1, B2, out, a, alpha, beta, vsrc, acol);
  } else {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    if (row < D)
      clenshaw_row_vs<T, S, false, SP, B2M, VS>(row, lane, rp, col, nullptr, V, B1, B2, out, a, alpha, beta, vsrc, acol);
  }
}

// Launch shape of a step over `rows` rows.  FP32 and pair-float steps, bound by their neighbour
// gathers, sweep the rows in order once there is more than one chunk of rows per CTA: one wave
// of CTAs strides over 256/G-row groups, so at any moment the whole GPU works inside a window of
// a few thousand consecutive rows.  A neighbour row behind the window was read a short while ago
// and is still in L1 or L2.  Hubbard L = 12 (6 up, 6 down), s = 64: 244 against 372 us per FP32
// step with one contiguous row range per CTA (there every CTA sits at its own place in a block
// larger than half of L2 and neighbours come from DRAM); XXZ L = 20, s = 32, whose block fits in
// L2: 25.2 against 26.7 us, L = 18: 9.4 against 10.0 us; the same bits in every shape.  FP64
// steps are bound by the FP64 pipe and keep one row per thread group.  cta_cap > 0 limits the
// CTAs per SM (the grid is then one wave of that many per SM: the sweep for FP32, a grid-stride
// loop for FP64), leaving SM thread slots and registers to a kernel of another solve running
// beside it.
struct StepShape {
  unsigned grid;
  int64_t rows_per_cta;
};
static int device_sms() {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  return nsm;
}
static int64_t device_l2_bytes() {
  static const int64_t l2 = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 126 << 20;
    }
    return (int64_t)v;
  }();
  return l2;
}
template <typename K>
static int kernel_occupancy(K kern) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0);
  return occ > 0 ? occ : 1;
}
template <typename T, int S>
static StepShape shape_for(int64_t rows, int cta_cap, int nsm, int occ) {
  using Sh = Shape<T, S>;
  const int per_sm = cta_cap > 0 ? std::min(occ, cta_cap) : occ;
  const int64_t waves = (int64_t)nsm * per_sm;
  if constexpr (!std::is_same_v<T, double>) {
    if (rows > waves * (256 / Sh::G)) return StepShape{(unsigned)waves, -1};   // sweep order
  }
  const int64_t classic = ceil_div(rows * Sh::G, 256);
  if (cta_cap > 0 && classic > waves) return StepShape{(unsigned)waves, -1};
  return StepShape{(unsigned)classic, 0};
}
template <typename T, int S, int SP, int B2M>
static StepShape step_shape(int64_t rows, int cta_cap = 0) {
  static const int nsm = device_sms();
  static const int occ = kernel_occupancy(clenshaw_step_kernel<T, S, SP, B2M>);
  return shape_for<T, S>(rows, cta_cap, nsm, occ);
}
template <typename T, int S, int SP, int B2M>
static StepShape qrem_shape(int64_t rows, int cta_cap = 0) {
  static const int nsm = device_sms();
  static const int occ = kernel_occupancy(qrem_step_kernel<T, S, SP, B2M>);
  return shape_for<T, S>(rows, cta_cap, nsm, occ);
}
template <typename T, int S, int SP, int B2M, int VS>
static StepShape cstruct_shape(int64_t rows, int cta_cap = 0) {
  static const int nsm = device_sms();
  static const int occ = kernel_occupancy(cstruct_step_kernel<T, S, SP, B2M, VS>);
  return shape_for<T, S>(rows, cta_cap, nsm, occ);
}

template <typename T, int S, int SP, int B2M>
static void launch_step_form(int64_t D, const int64_t* rp, const int32_t* col, const T* val, const T* V, const T* B1,
                             const T* B2, T* out, T a, T alpha, T beta, cudaStream_t st, int cta_cap, const T* acol) {
  const StepShape sh = step_shape<T, S, SP, B2M>(D, cta_cap);
  clenshaw_step_kernel<T, S, SP, B2M><<<sh.grid, 256, 0, st>>>(D, rp, col, val, V, B1, B2, out, a, alpha, beta,
                                                              sh.rows_per_cta, acol);
}

template <typename T, int S>
static pf_status launch_step_s(int64_t D, const int64_t* rp, const int32_t* col, const T* val, const T* V, const T* B1,
                               const T* B2, T* out, T a, T alpha, T beta, cudaStream_t st, int cap, const T* acol) {
  const bool spmm = alpha != T(0);
  const bool hb2 = beta != T(0);
  if (spmm && hb2) launch_step_form<T, S, 1, 1>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  else if (spmm) launch_step_form<T, S, 1, 0>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  else if (hb2) launch_step_form<T, S, 0, 1>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  else launch_step_form<T, S, 0, 0>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  PF_LAUNCH_CHECK("clenshaw_step_kernel");
  return PF_OK;
}

template <typename T>
static pf_status launch_step(int s, int64_t D, const int64_t* rp, const int32_t* col, const T* val, const T* V,
                             const T* B1, const T* B2, T* out, T a, T alpha, T beta, cudaStream_t st, int cap,
                             const T* acol) {
  switch (s) {
    case 1: return launch_step_s<T, 1>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 2: return launch_step_s<T, 2>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 4: return launch_step_s<T, 4>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 8: return launch_step_s<T, 8>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 16: return launch_step_s<T, 16>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 32: return launch_step_s<T, 32>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 64: return launch_step_s<T, 64>(D, rp, col, val, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  }
  return PF_EINVAL;
}

static bool valid_s(int s) { return s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32 || s == 64; }

pf_status clenshaw_step_raw(int64_t D, const int64_t* row_ptr, const int32_t* col, const void* val, int prec, int s,
                            const void* V, const void* B1, const void* B2, void* out, double a, double alpha,
                            double beta, cudaStream_t st, int cta_cap, const void* acol) {
  if (!valid_s(s) || D <= 0 || !V || !out) return PF_EINVAL;
  if (alpha != 0.0 && (!B1 || !val)) return PF_EINVAL;
  if (beta != 0.0 && !B2) return PF_EINVAL;
  if (beta != 0.0 && beta != 1.0) return PF_EINVAL;
  if (prec == PF_F64)
    return launch_step<double>(s, D, row_ptr, col, (const double*)val, (const double*)V, (const double*)B1,
                               (const double*)B2, (double*)out, a, alpha, beta, st, cta_cap, (const double*)acol);
  if (prec == PF_F32)
    return launch_step<float>(s, D, row_ptr, col, (const float*)val, (const float*)V, (const float*)B1,
                              (const float*)B2, (float*)out, (float)a, (float)alpha, (float)beta, st, cta_cap,
                              (const float*)acol);
  if (prec == PF_DF64 && !acol)
    return launch_step<df2>(s, D, row_ptr, col, (const df2*)val, (const df2*)V, (const df2*)B1, (const df2*)B2,
                            (df2*)out, df2(a), df2(alpha), df2(beta), st, cta_cap, nullptr);
  return PF_EINVAL;
}

// Structured-mapping step launches (QREM bit flips, or XXZ constant off-diagonal): same shapes,
// validation and operands as the CSR step.  The structure argument is L for QREM and the CSR
// (row pointers, columns) for XXZ.
enum { MAP_QREM = 0, MAP_XXZ = 1, MAP_QSUN = 2 };
template <int KIND, typename T, int S, int SP, int B2M>
static void launch_struct_form(const Ham* H, const ValSrc<T>& vs, const T* V, const T* B1, const T* B2, T* out, T a,
                               T alpha, T beta, cudaStream_t st, int cap, const T* acol) {
  const int64_t D = H->D;
  if constexpr (KIND == MAP_QREM) {
    const StepShape sh = qrem_shape<T, S, SP, B2M>(D, cap);
    qrem_step_kernel<T, S, SP, B2M><<<sh.grid, 256, 0, st>>>(D, H->m.L, vs.diag, vs.g, V, B1, B2, out, a, alpha, beta,
                                                            sh.rows_per_cta, acol);
  } else {
    constexpr int VS = KIND == MAP_XXZ ? 1 : 2;
    const StepShape sh = cstruct_shape<T, S, SP, B2M, VS>(D, cap);
    cstruct_step_kernel<T, S, SP, B2M, VS><<<sh.grid, 256, 0, st>>>(D, H->row_ptr, H->col, vs, V, B1, B2, out, a,
                                                                    alpha, beta, sh.rows_per_cta, acol);
  }
}
template <int KIND, typename T, int S>
static pf_status launch_struct_s(const Ham* H, const ValSrc<T>& vs, const T* V, const T* B1, const T* B2, T* out,
                                 T a, T alpha, T beta, cudaStream_t st, int cap, const T* acol) {
  const bool spmm = alpha != T(0);
  const bool hb2 = beta != T(0);
  if (spmm && hb2) launch_struct_form<KIND, T, S, 1, 1>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  else if (spmm) launch_struct_form<KIND, T, S, 1, 0>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  else if (hb2) launch_struct_form<KIND, T, S, 0, 1>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  else launch_struct_form<KIND, T, S, 0, 0>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  PF_LAUNCH_CHECK(KIND == MAP_QREM ? "qrem_step_kernel" : "cstruct_step_kernel");
  return PF_OK;
}
template <int KIND, typename T>
static pf_status launch_struct(int s, const Ham* H, const ValSrc<T>& vs, const T* V, const T* B1, const T* B2, T* out,
                               T a, T alpha, T beta, cudaStream_t st, int cap, const T* acol) {
  switch (s) {
    case 1: return launch_struct_s<KIND, T, 1>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 2: return launch_struct_s<KIND, T, 2>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 4: return launch_struct_s<KIND, T, 4>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 8: return launch_struct_s<KIND, T, 8>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 16: return launch_struct_s<KIND, T, 16>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 32: return launch_struct_s<KIND, T, 32>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
    case 64: return launch_struct_s<KIND, T, 64>(H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  }
  return PF_EINVAL;
}
template <typename T>
static pf_status launch_structured(const Ham* H, int s, const ValSrc<T>& vs, const T* V, const T* B1, const T* B2,
                                   T* out, T a, T alpha, T beta, cudaStream_t st, int cap, const T* acol) {
  if (H->m.kind == PF_MODEL_QREM)
    return launch_struct<MAP_QREM, T>(s, H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  if (H->m.kind == PF_MODEL_QSUN)
    return launch_struct<MAP_QSUN, T>(s, H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
  return launch_struct<MAP_XXZ, T>(s, H, vs, V, B1, B2, out, a, alpha, beta, st, cap, acol);
}

// One step of H~ through the handle's mapping: the CSR arrays, or the structured rows (QREM bit
// flips; XXZ constant off-diagonal).
pf_status ham_step(const Ham* H, int prec, int s, const void* V, const void* B1, const void* B2, void* out,
                   double a, double alpha, double beta, cudaStream_t st, int cta_cap, const void* acol) {
  // XXZ and Hubbard: only the FP32 step takes the structured form (XXZ L = 20, s = 32: 26.7
  // against 28.8 us); FP64 (bound by its pipe, 145.4 against 145.6 us) and pair-float (73.5
  // against 73.0 us) keep the CSR form.  The bits are the same either way.
  const bool csr_form = H->mapping != PF_MAP_STRUCTURED || !H->diag_t ||
                        ((H->m.kind == PF_MODEL_XXZ || H->m.kind == PF_MODEL_QSUN || H->m.kind == PF_MODEL_HUBBARD) &&
                         prec != PF_F32) ||
                        (H->m.kind == PF_MODEL_QSUN && !H->qtab_t);
  if (csr_form)
    return clenshaw_step_raw(H->D, H->row_ptr, H->col, ham_vals(H, prec), prec, s, V, B1, B2, out, a, alpha, beta,
                             st, cta_cap, acol);
  if (!valid_s(s) || !V || !out) return PF_EINVAL;
  if (alpha != 0.0 && !B1) return PF_EINVAL;
  if (beta != 0.0 && !B2) return PF_EINVAL;
  if (beta != 0.0 && beta != 1.0) return PF_EINVAL;
  const int L = H->m.L, N = H->m.N;
  if (prec == PF_F64) {
    ValSrc<double> vs;
    vs.diag = H->diag_t; vs.g = H->off_t; vs.tab = H->qtab_t; vs.coef = H->qtab_t ? H->qtab_t + H->qtab_n : nullptr;
    vs.L = L; vs.N = N;
    return launch_structured<double>(H, s, vs, (const double*)V, (const double*)B1, (const double*)B2, (double*)out,
                                     a, alpha, beta, st, cta_cap, (const double*)acol);
  }
  if (prec == PF_F32) {
    ValSrc<float> vs;
    vs.diag = H->diag32; vs.g = (float)H->off_t; vs.tab = H->qtab32; vs.coef = H->qtab32 ? H->qtab32 + H->qtab_n : nullptr;
    vs.L = L; vs.N = N;
    return launch_structured<float>(H, s, vs, (const float*)V, (const float*)B1, (const float*)B2, (float*)out,
                                    (float)a, (float)alpha, (float)beta, st, cta_cap, (const float*)acol);
  }
  if (prec == PF_DF64 && !acol) {
    ValSrc<df2> vs;
    const df2* tab = reinterpret_cast<const df2*>(H->qtab_df);
    vs.diag = reinterpret_cast<const df2*>(H->diag_df); vs.g = df2(H->off_t); vs.tab = tab;
    vs.coef = tab ? tab + H->qtab_n : nullptr;
    vs.L = L; vs.N = N;
    return launch_structured<df2>(H, s, vs, (const df2*)V, (const df2*)B1, (const df2*)B2, (df2*)out, df2(a),
                                  df2(alpha), df2(beta), st, cta_cap, nullptr);
  }
  return PF_EINVAL;
}

// K-step recurrence.  b_i lives in aux[i & 1]: step i reads b_{i+1} = aux[(i+1)&1] and
// overwrites b_{i+2} (= aux[i&1]) with b_i.  colcoef (device, (K+1) x s values in the filter
// precision, FP64 or FP32 only), when not null, gives every column its own coefficients: step i
// uses row i of the table in place of coeffs[i] (the residual-correction form of the refinement).
pf_status filter_apply_raw(const Ham* H, int prec, int s, const void* V, void* W, const double* coeffs,
                           const void* colcoef, int K, void* aux0, void* aux1, cudaStream_t st, int cta_cap) {
  if (K < 1 || (!coeffs && !colcoef)) return PF_EINVAL;
  if (colcoef && prec != PF_F64 && prec != PF_F32) return PF_EINVAL;
  const size_t w = prec_bytes(prec);
  auto ac = [&](int i) -> const void* {
    return colcoef ? static_cast<const void*>(static_cast<const char*>(colcoef) + (size_t)i * s * w) : nullptr;
  };
  auto a = [&](int i) { return colcoef ? 0.0 : coeffs[i]; };
  void* aux[2] = {aux0, aux1};
  // i = K: b_K = a_K V
  PF_TRY(ham_step(H, prec, s, V, nullptr, nullptr, aux[K & 1], a(K), 0.0, 0.0, st, cta_cap, ac(K)));
  for (int i = K - 1; i >= 1; --i) {
    const double beta = (i == K - 1) ? 0.0 : 1.0;
    PF_TRY(ham_step(H, prec, s, V, aux[(i + 1) & 1], aux[i & 1], aux[i & 1], a(i), 2.0, beta, st, cta_cap, ac(i)));
  }
  // P V = a_0 V + H~ b_1 - b_2
  const double beta = (K >= 2) ? 1.0 : 0.0;
  PF_TRY(ham_step(H, prec, s, V, aux[1], aux[0], W, a(0), 1.0, beta, st, cta_cap, ac(0)));
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

// Operands of recurrence index i of one item, as in filter_apply_raw: b_i lives in aux[i & 1].
template <typename T>
__device__ __forceinline__ void step_operands(const BatchItemDev& it, int i, const T*& B1, const T*& B2, T*& out,
                                              T& alpha, T& beta) {
  T* const a0 = (T*)it.aux0;
  T* const a1 = (T*)it.aux1;
  T* const cur = (i & 1) ? a1 : a0;    // aux[i & 1]
  T* const nxt = (i & 1) ? a0 : a1;    // aux[(i + 1) & 1]
  const int K = it.K;
  if (i == K) {
    alpha = T(0); beta = T(0); B1 = nullptr; B2 = nullptr; out = cur;
  } else if (i >= 1) {
    alpha = T(2); beta = (i == K - 1) ? T(0) : T(1);
    B1 = nxt; B2 = cur; out = cur;
  } else {
    alpha = T(1); beta = (K >= 2) ? T(1) : T(0);
    B1 = a1; B2 = a0; out = (T*)it.W;
  }
}

__device__ __forceinline__ int find_item(const BatchItemDev* __restrict__ items, int n, int64_t grow) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].row0 <= grow) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Sweep step t over all items' rows (items may differ in K).  UNI = 1: every item has the
// same K (all t0 = 0), so the step's form (SP, B2M) is the same for all and fixed at compile
// time, as in clenshaw_step_kernel.  rows_per_cta as in clenshaw_step_kernel (< 0: sweep order
// over row groups; 0: one row group per thread group).
template <typename T, int S, int SP, int B2M>
__global__ void __launch_bounds__(256, 4) clenshaw_batch_kernel(const BatchItemDev* __restrict__ items, int n, int t,
                                                             int64_t total_rows, int64_t rows_per_cta) {
  using Sh = Shape<T, S>;
  constexpr int G = Sh::G;
  const int lane = (int)(threadIdx.x % G);
  int64_t r0, r1, stride;
  if (rows_per_cta < 0) {   // sweep order: one wave of CTAs strides over row groups
    r0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    r1 = total_rows;
    stride = (int64_t)gridDim.x * (256 / G);
  } else {
    r0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    r1 = r0 + 1 < total_rows ? r0 + 1 : total_rows;
    stride = 1;
  }
  for (int64_t grow = r0; grow < r1; grow += stride) {
    const BatchItemDev& it = items[find_item(items, n, grow)];
    if (t < it.t0) continue;
    const int i = it.K - (t - it.t0);
    const T* B1;
    const T* B2;
    T* out;
    T alpha, beta;
    step_operands<T>(it, i, B1, B2, out, alpha, beta);
    clenshaw_row<T, S, false, SP, B2M>(grow - it.row0, lane, it.rp, it.col, (const T*)it.val, (const T*)it.V, B1,
                                       B2, out, load_coeff<T>(it.coeffs + i), alpha, beta);
  }
}

// Persistent form for small items: one thread-block cluster per item (csize CTAs, its rows
// split evenly) runs the item's whole recurrence, K+1 steps, in one launch.  Between steps
// the cluster meets at the hardware cluster barrier (arrive.release / wait.acquire), which
// orders the step's global stores before the next step's loads; b blocks are read with
// L2-only loads so no SM reuses a line it cached before the rewrite.  With csize = 1 the
// barrier is __syncthreads().  No spin-waits: both barriers are hardware barriers.
#define PF_PERSIST_NT 512
template <typename T, int S, bool CLUSTER>
__global__ void __launch_bounds__(PF_PERSIST_NT) clenshaw_persistent_kernel(const BatchItemDev* __restrict__ items,
                                                                           int n) {
  using Sh = Shape<T, S>;
  constexpr int G = Sh::G, ROWS = PF_PERSIST_NT / G;
  unsigned csize = 1, crank = 0, cid = blockIdx.x;
  if constexpr (CLUSTER) {
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cid));
  }
  if ((int)cid >= n) return;   // uniform over the cluster
  const BatchItemDev& it = items[cid];
  const int64_t per = (it.D + csize - 1) / csize;
  const int64_t r0 = crank * per;
  const int64_t r1 = r0 + per < it.D ? r0 + per : it.D;
  const int lane = threadIdx.x % G;
  const T* __restrict__ val = (const T*)it.val;
  const T* __restrict__ V = (const T*)it.V;
  for (int i = it.K; i >= 0; --i) {
    const T* B1;
    const T* B2;
    T* out;
    T alpha, beta;
    step_operands<T>(it, i, B1, B2, out, alpha, beta);
    const T a = load_coeff<T>(it.coeffs + i);
    for (int64_t row = r0 + threadIdx.x / G; row < r1; row += ROWS)
      clenshaw_row<T, S, true, -1, -1>(row, lane, it.rp, it.col, val, V, B1, B2, out, a, alpha, beta);
    if constexpr (CLUSTER) {
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
      __syncthreads();
    }
  }
}

template <typename T, int S>
static pf_status launch_persistent_s(const BatchItemDev* items, int n, int csize, cudaStream_t st) {
  if (csize <= 1) {
    clenshaw_persistent_kernel<T, S, false><<<n, PF_PERSIST_NT, 0, st>>>(items, n);
    PF_LAUNCH_CHECK("clenshaw_persistent_kernel");
    return PF_OK;
  }
  auto kern = clenshaw_persistent_kernel<T, S, true>;
  if (csize > 8) PF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * csize), 1, 1);
  cfg.blockDim = dim3(PF_PERSIST_NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PF_COUNT(1);
  PF_CUDA(cudaLaunchKernelEx(&cfg, kern, items, n));
  return PF_OK;
}

// Step t of a sweep: its kernel entry and launch shape.  uniform: all items share K, so the
// step's (SP, B2M) is known: t = 0 is b_K (no SpMM, no B2), t = 1 has no B2 (b_{K+1} = 0),
// the last step (i = 0) has B2 when K >= 2; the generic form decides per item at run time.
template <typename T, int S>
static void* sweep_fn(bool uniform, int t, int K) {
  if (!uniform) return (void*)clenshaw_batch_kernel<T, S, -1, -1>;
  const int i = K - t;
  if (i == K) return (void*)clenshaw_batch_kernel<T, S, 0, 0>;
  if (i == K - 1 || (i == 0 && K < 2)) return (void*)clenshaw_batch_kernel<T, S, 1, 0>;
  return (void*)clenshaw_batch_kernel<T, S, 1, 1>;
}

template <typename T, int S>
static StepShape sweep_shape(int64_t rows) { return step_shape<T, S, 1, 1>(rows); }

template <typename T, int S>
static pf_status launch_batch_s(const BatchItemDev* items, int n, int T_steps, int64_t total_rows, bool uniform,
                                cudaStream_t st) {
  const StepShape sh = sweep_shape<T, S>(total_rows);
  for (int t = 0; t < T_steps; ++t) {
    void* fn = sweep_fn<T, S>(uniform, t, T_steps - 1);
    int nn = n, tt = t;
    int64_t rr = total_rows, rpc = sh.rows_per_cta;
    void* args[] = {(void*)&items, (void*)&nn, (void*)&tt, (void*)&rr, (void*)&rpc};
    PF_CUDA(cudaLaunchKernel(fn, dim3(sh.grid), dim3(256), args, 0, st));
    PF_COUNT(1);
  }
  return PF_OK;
}

template <typename T>
static void* sweep_fn_s(int s, bool uniform, int t, int K) {
  switch (s) {
    case 1: return sweep_fn<T, 1>(uniform, t, K);
    case 2: return sweep_fn<T, 2>(uniform, t, K);
    case 4: return sweep_fn<T, 4>(uniform, t, K);
    case 8: return sweep_fn<T, 8>(uniform, t, K);
    case 16: return sweep_fn<T, 16>(uniform, t, K);
    case 32: return sweep_fn<T, 32>(uniform, t, K);
    case 64: return sweep_fn<T, 64>(uniform, t, K);
  }
  return nullptr;
}

template <typename T>
static StepShape sweep_shape_s(int s, int64_t rows) {
  switch (s) {
    case 1: return sweep_shape<T, 1>(rows);
    case 2: return sweep_shape<T, 2>(rows);
    case 4: return sweep_shape<T, 4>(rows);
    case 8: return sweep_shape<T, 8>(rows);
    case 16: return sweep_shape<T, 16>(rows);
    case 32: return sweep_shape<T, 32>(rows);
    case 64: return sweep_shape<T, 64>(rows);
  }
  return StepShape{0, 0};
}

static int lanes_per_row(int prec, int s) {   // Shape<T, s>::G
  const int E = prec == PF_F64 ? (s >= 64 ? s / 32 : 1) : prec == PF_DF64 ? (s >= PF_DF_E ? PF_DF_E : s)
                                                                          : (s * 4 >= 16 ? 4 : s);
  return s / E;
}

SweepGraph::~SweepGraph() { reset(); }
void SweepGraph::reset() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  T = 0;
}

// The T launches of one sweep as a chain of kernel nodes.  The nodes read the item table from
// device memory at run time, so one instantiated graph serves every sweep with the same
// table address, item count, step count, row total and uniformity; only the table contents
// change between launches.
static pf_status sweep_graph_launch(SweepGraph& g, int prec, int s, const void* table, int n, int T, int64_t rows,
                                    bool uniform, cudaStream_t st) {
  if (!(g.exec && g.prec == prec && g.s == s && g.table == table && g.n == n && g.T == T && g.rows == rows &&
        g.uniform == uniform)) {
    g.reset();
    PF_CUDA(cudaGraphCreate(&g.graph, 0));
    const StepShape sh = prec == PF_F64 ? sweep_shape_s<double>(s, rows)
                         : prec == PF_DF64 ? sweep_shape_s<df2>(s, rows) : sweep_shape_s<float>(s, rows);
    cudaGraphNode_t prev = nullptr;
    for (int t = 0; t < T; ++t) {
      void* fn = prec == PF_F64    ? sweep_fn_s<double>(s, uniform, t, T - 1)
                 : prec == PF_DF64 ? sweep_fn_s<df2>(s, uniform, t, T - 1)
                                   : sweep_fn_s<float>(s, uniform, t, T - 1);
      if (!fn || sh.grid == 0) return PF_EINVAL;
      const BatchItemDev* items = static_cast<const BatchItemDev*>(table);
      int nn = n, tt = t;
      int64_t rr = rows, rpc = sh.rows_per_cta;
      void* args[] = {(void*)&items, (void*)&nn, (void*)&tt, (void*)&rr, (void*)&rpc};
      cudaKernelNodeParams kp = {};
      kp.func = fn;
      kp.gridDim = dim3(sh.grid, 1, 1);
      kp.blockDim = dim3(256, 1, 1);
      kp.sharedMemBytes = 0;
      kp.kernelParams = args;
      kp.extra = nullptr;
      cudaGraphNode_t node;
      PF_CUDA(cudaGraphAddKernelNode(&node, g.graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
      prev = node;
    }
    PF_CUDA(cudaGraphInstantiate(&g.exec, g.graph, 0));
    g.prec = prec;
    g.s = s;
    g.table = table;
    g.n = n;
    g.T = T;
    g.rows = rows;
    g.uniform = uniform;
  }
  PF_COUNT(T);
  PF_CUDA(cudaGraphLaunch(g.exec, st));
  return PF_OK;
}

pf_status filter_sweep(const std::vector<FilterItem>& items, void* table_dev, size_t table_bytes, void* table_host,
                       cudaStream_t st, int csize, SweepGraph* graph) {
  const int n = (int)items.size();
  if (n == 0) return PF_OK;
  if ((size_t)n * sizeof(BatchItemDev) > table_bytes) return PF_EINVAL;
  const int prec = items[0].prec, s = items[0].s;
  if (!valid_s(s) || !valid_prec(prec) || csize < 0 || csize > 16) return PF_EINVAL;
  int T = 0;
  bool uniform = true;
  for (const auto& it : items) {
    if (it.prec != prec || it.s != s || it.K < 1 || !it.coeffs_dev) return PF_EINVAL;
    T = std::max(T, it.K + 1);
    uniform = uniform && it.K == items[0].K;
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
    b.val = ham_vals(it.H, prec);
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
  if (csize >= 1) {
#define PF_PERSIST_CASE(TT, SS) \
  case SS: return launch_persistent_s<TT, SS>(d, n, csize, st);
    if (prec == PF_F64) {
      switch (s) { PF_PERSIST_CASE(double, 1) PF_PERSIST_CASE(double, 2) PF_PERSIST_CASE(double, 4)
                   PF_PERSIST_CASE(double, 8) PF_PERSIST_CASE(double, 16) PF_PERSIST_CASE(double, 32)
                   PF_PERSIST_CASE(double, 64) }
    } else if (prec == PF_DF64) {
      switch (s) { PF_PERSIST_CASE(df2, 1) PF_PERSIST_CASE(df2, 2) PF_PERSIST_CASE(df2, 4)
                   PF_PERSIST_CASE(df2, 8) PF_PERSIST_CASE(df2, 16) PF_PERSIST_CASE(df2, 32)
                   PF_PERSIST_CASE(df2, 64) }
    } else {
      switch (s) { PF_PERSIST_CASE(float, 1) PF_PERSIST_CASE(float, 2) PF_PERSIST_CASE(float, 4)
                   PF_PERSIST_CASE(float, 8) PF_PERSIST_CASE(float, 16) PF_PERSIST_CASE(float, 32)
                   PF_PERSIST_CASE(float, 64) }
    }
#undef PF_PERSIST_CASE
    return PF_EINVAL;
  }
  if (graph) return sweep_graph_launch(*graph, prec, s, table_dev, n, T, row0, uniform, st);
  if (prec == PF_F64) {
    switch (s) {
      case 1: return launch_batch_s<double, 1>(d, n, T, row0, uniform, st);
      case 2: return launch_batch_s<double, 2>(d, n, T, row0, uniform, st);
      case 4: return launch_batch_s<double, 4>(d, n, T, row0, uniform, st);
      case 8: return launch_batch_s<double, 8>(d, n, T, row0, uniform, st);
      case 16: return launch_batch_s<double, 16>(d, n, T, row0, uniform, st);
      case 32: return launch_batch_s<double, 32>(d, n, T, row0, uniform, st);
      case 64: return launch_batch_s<double, 64>(d, n, T, row0, uniform, st);
    }
  } else if (prec == PF_DF64) {
    switch (s) {
      case 1: return launch_batch_s<df2, 1>(d, n, T, row0, uniform, st);
      case 2: return launch_batch_s<df2, 2>(d, n, T, row0, uniform, st);
      case 4: return launch_batch_s<df2, 4>(d, n, T, row0, uniform, st);
      case 8: return launch_batch_s<df2, 8>(d, n, T, row0, uniform, st);
      case 16: return launch_batch_s<df2, 16>(d, n, T, row0, uniform, st);
      case 32: return launch_batch_s<df2, 32>(d, n, T, row0, uniform, st);
      case 64: return launch_batch_s<df2, 64>(d, n, T, row0, uniform, st);
    }
  } else {
    switch (s) {
      case 1: return launch_batch_s<float, 1>(d, n, T, row0, uniform, st);
      case 2: return launch_batch_s<float, 2>(d, n, T, row0, uniform, st);
      case 4: return launch_batch_s<float, 4>(d, n, T, row0, uniform, st);
      case 8: return launch_batch_s<float, 8>(d, n, T, row0, uniform, st);
      case 16: return launch_batch_s<float, 16>(d, n, T, row0, uniform, st);
      case 32: return launch_batch_s<float, 32>(d, n, T, row0, uniform, st);
      case 64: return launch_batch_s<float, 64>(d, n, T, row0, uniform, st);
    }
  }
  return PF_EINVAL;
}

// ------------------------------------------------------------------ captured filter applications
// One filter application with fixed operands (V, W, auxiliaries, coefficients) captured once
// from filter_apply_raw into a CUDA graph, then replayed with one launch call.  Used where a
// host thread drives many solves at once: a whole K-step recurrence is queued by a single
// call, so the thread never stalls on a full launch queue.
FilterGraph::~FilterGraph() { reset(); }
void FilterGraph::reset() {
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  exec = nullptr;
  graph = nullptr;
  K = -1;
}

// Settles the step kernels' launch-shape queries (occupancy) before a capture begins.
template <typename T, int S>
static void prepare_shapes_s() {
  step_shape<T, S, 0, 0>(1);
  step_shape<T, S, 1, 0>(1);
  step_shape<T, S, 0, 1>(1);
  step_shape<T, S, 1, 1>(1);
  qrem_shape<T, S, 0, 0>(1);
  qrem_shape<T, S, 1, 0>(1);
  qrem_shape<T, S, 0, 1>(1);
  qrem_shape<T, S, 1, 1>(1);
  cstruct_shape<T, S, 0, 0, 1>(1);
  cstruct_shape<T, S, 1, 0, 1>(1);
  cstruct_shape<T, S, 0, 1, 1>(1);
  cstruct_shape<T, S, 1, 1, 1>(1);
  cstruct_shape<T, S, 0, 0, 2>(1);
  cstruct_shape<T, S, 1, 0, 2>(1);
  cstruct_shape<T, S, 0, 1, 2>(1);
  cstruct_shape<T, S, 1, 1, 2>(1);
}
template <typename T>
static void prepare_shapes(int s) {
  switch (s) {
    case 1: prepare_shapes_s<T, 1>(); break;
    case 2: prepare_shapes_s<T, 2>(); break;
    case 4: prepare_shapes_s<T, 4>(); break;
    case 8: prepare_shapes_s<T, 8>(); break;
    case 16: prepare_shapes_s<T, 16>(); break;
    case 32: prepare_shapes_s<T, 32>(); break;
    case 64: prepare_shapes_s<T, 64>(); break;
  }
}

pf_status filter_graph_launch(FilterGraph& g, const FilterItem& it, cudaStream_t st) {
  const double a0 = it.coeffs_host ? it.coeffs_host[0] : 0.0;
  const double aK = it.coeffs_host ? it.coeffs_host[it.K] : 0.0;
  if (!(g.exec && g.K == it.K && g.V == it.V && g.W == it.W && g.aux0 == it.aux0 && g.aux1 == it.aux1 &&
        g.prec == it.prec && g.s == it.s && g.H == it.H && g.a0 == a0 && g.aK == aK && g.cap == it.cta_cap &&
        g.colcoef == it.colcoef)) {
    g.reset();
    if ((!it.coeffs_host && !it.colcoef) || it.K < 1) return PF_EINVAL;
    if (it.prec == PF_F64) prepare_shapes<double>(it.s);
    else if (it.prec == PF_DF64) prepare_shapes<df2>(it.s);
    else prepare_shapes<float>(it.s);
    cudaStream_t cap = nullptr;
    PF_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    const long long before = g_kernel_launches.load();
    pf_status rc = PF_OK;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      rc = filter_apply_raw(it.H, it.prec, it.s, it.V, it.W, it.coeffs_host, it.colcoef, it.K, it.aux0, it.aux1, cap,
                            it.cta_cap);
      e = cudaStreamEndCapture(cap, &g.graph);
    }
    g_kernel_launches.store(before);   // capture is not execution
    cudaStreamDestroy(cap);
    if (rc == PF_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (rc != PF_OK || e != cudaSuccess) {
      // no graph: the same launches go to the stream one by one
      g.reset();
      cudaGetLastError();
      return filter_apply_raw(it.H, it.prec, it.s, it.V, it.W, it.coeffs_host, it.colcoef, it.K, it.aux0, it.aux1, st,
                              it.cta_cap);
    }
    g.K = it.K;
    g.V = it.V;
    g.W = it.W;
    g.aux0 = it.aux0;
    g.aux1 = it.aux1;
    g.prec = it.prec;
    g.s = it.s;
    g.H = it.H;
    g.a0 = a0;
    g.aK = aK;
    g.cap = it.cta_cap;
    g.colcoef = it.colcoef;
  }
  PF_COUNT(it.K + 1);
  PF_CUDA(cudaGraphLaunch(g.exec, st));
  return PF_OK;
}

// ------------------------------------------------------------------ autotuner
// Execution form of a group of n items of one shape.  Measured once per (device, D, nnz,
// precision, s) on scratch blocks (the caller's data is untouched), over min(K, 48) + 1 steps:
//   raw_us      one item alone, one launch per step (filter_apply_raw);
//   sweep_us    the per-step sweep over r copies of the item (r fills the GPU);
//   persist_us  one item in the persistent kernel with clusters of c = 1, 2, 4, 8, 16 CTAs,
//               of which slots[c] run at once.
// choose_form() then predicts the per-step time of the whole group for each form and takes
// the fastest: raw (n = 1) raw_us; sweep, interpolated between raw_us (one item) and sweep_us
// (r items) and proportional beyond r; persistent c, persist_us x ceil(n / slots).  Items
// with more than 64 rows per thread of a 16-CTA cluster are not measured: they take the
// sweep (or the plain recurrence when alone).
namespace {
struct TuneKey {
  int dev, prec, s;
  int64_t D, nnz;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, prec, s, D, nnz) < std::tie(o.dev, o.prec, o.s, o.D, o.nnz);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune;
}  // namespace

static pf_status time_ms(cudaStream_t st, const std::function<pf_status()>& f, int reps, double* ms) {
  cudaEvent_t a, b;
  PF_CUDA(cudaEventCreate(&a));
  PF_CUDA(cudaEventCreate(&b));
  pf_status rc = f();   // warm-up
  if (rc == PF_OK) {
    cudaEventRecord(a, st);
    for (int r = 0; r < reps && rc == PF_OK; ++r) rc = f();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float t = 0;
    cudaEventElapsedTime(&t, a, b);
    *ms = t / reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return rc;
}

template <typename T, int S>
static int persist_slots_s(int c, int nsm) {
  if (c <= 1) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, clenshaw_persistent_kernel<T, S, false>, PF_PERSIST_NT, 0);
    return nsm * std::max(occ, 1);
  }
  auto kern = clenshaw_persistent_kernel<T, S, true>;
  if (c > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c, 1, 1);
  cfg.blockDim = dim3(PF_PERSIST_NT, 1, 1);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return std::max(1, nsm / c);
  }
  return std::max(n, 1);
}

template <typename T>
static int persist_slots(int s, int c, int nsm) {
  switch (s) {
    case 1: return persist_slots_s<T, 1>(c, nsm);
    case 2: return persist_slots_s<T, 2>(c, nsm);
    case 4: return persist_slots_s<T, 4>(c, nsm);
    case 8: return persist_slots_s<T, 8>(c, nsm);
    case 16: return persist_slots_s<T, 16>(c, nsm);
    case 32: return persist_slots_s<T, 32>(c, nsm);
    case 64: return persist_slots_s<T, 64>(c, nsm);
  }
  return 1;
}

int choose_form(const TuneResult& tr, int n, double* predicted_us) {
  double best = 0;
  int form = 0;
  if (tr.raw_us > 0) {
    if (n <= 1) {
      best = tr.raw_us;
    } else if (n <= tr.sweep_copies) {
      best = tr.raw_us + (tr.sweep_us - tr.raw_us) * (double)(n - 1) / std::max(1, tr.sweep_copies - 1);
    } else {
      best = tr.sweep_us * (double)n / tr.sweep_copies;
    }
    const int cs[5] = {1, 2, 4, 8, 16};
    for (int k = 0; k < 5; ++k) {
      if (tr.persist_us[k] <= 0) continue;
      const double t = tr.persist_us[k] * (double)ceil_div(n, std::max(1, tr.slots[k]));
      if (t < best) {
        best = t;
        form = cs[k];
      }
    }
  }
  if (predicted_us) *predicted_us = best;
  return form;
}

pf_status tune_item(const FilterItem& it, cudaStream_t st, TuneResult* out) {
  int dev = 0;
  PF_CUDA(cudaGetDevice(&dev));
  const TuneKey key{dev, it.prec, it.s, it.H->D, it.H->nnz};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto f = g_tune.find(key);
    if (f != g_tune.end()) {
      *out = f->second;
      return PF_OK;
    }
  }
  TuneResult res;
  const int G = lanes_per_row(it.prec, it.s);
  const int64_t D = it.H->D;
  int nsm = 148;
  PF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const bool small = D * G <= (int64_t)16 * PF_PERSIST_NT * 64;
  if (small) {
    const size_t w = prec_bytes(it.prec);
    const size_t blk = (((size_t)D * it.s * w) + 255) & ~(size_t)255;
    const int Kt = std::min(it.K, 48);
    // r copies fill the GPU in the sweep (about 8 resident 256-thread CTAs per SM)
    const int r = (int)std::max<int64_t>(2, std::min<int64_t>(64, ceil_div((int64_t)nsm * 8 * 256, D * G)));
    DevBuf scratch, table;
    PF_TRY(scratch.alloc(blk * 3 * r, st));
    PF_TRY(table.alloc(filter_sweep_table_bytes(r), st));
    std::vector<FilterItem> one(1, it), many(r, it);
    for (int j = 0; j < r; ++j) {
      unsigned char* b = scratch.as<unsigned char>() + blk * 3 * j;
      many[j].aux0 = b;
      many[j].aux1 = b + blk;
      many[j].W = b + 2 * blk;
      many[j].K = Kt;
    }
    one[0] = many[0];
    std::vector<double> ch(Kt + 1);
    PF_CUDA(cudaMemcpyAsync(ch.data(), it.coeffs_dev, (Kt + 1) * 8, cudaMemcpyDeviceToHost, st));
    PF_CUDA(cudaStreamSynchronize(st));
    for (double& c : ch) c = coeff_value_host(it.prec, c);
    std::vector<unsigned char> th(filter_sweep_table_bytes(r));
    double ms = 0;
    const FilterItem& o = one[0];
    PF_TRY(time_ms(st, [&] {
      return filter_apply_raw(o.H, o.prec, o.s, o.V, o.W, ch.data(), nullptr, Kt, o.aux0, o.aux1, st);
    }, 3, &ms));
    res.raw_us = 1e3 * ms / (Kt + 1);
    PF_TRY(time_ms(st, [&] { return filter_sweep(many, table.p, table.bytes, th.data(), st, 0, nullptr); }, 3, &ms));
    res.sweep_us = 1e3 * ms / (Kt + 1);
    res.sweep_copies = r;
    const int cs[5] = {1, 2, 4, 8, 16};
    for (int k = 0; k < 5; ++k) {
      const int c = cs[k];
      if (c > 1 && D < (int64_t)c * (PF_PERSIST_NT / G)) break;   // fewer rows than one pass of c CTAs
      pf_status rc = time_ms(st, [&] { return filter_sweep(one, table.p, table.bytes, th.data(), st, c, nullptr); },
                             3, &ms);
      if (rc != PF_OK) {   // a cluster shape the device refuses: clear the error and stop growing
        cudaGetLastError();
        break;
      }
      res.persist_us[k] = 1e3 * ms / (Kt + 1);
      res.slots[k] = it.prec == PF_F64    ? persist_slots<double>(it.s, c, nsm)
                     : it.prec == PF_DF64 ? persist_slots<df2>(it.s, c, nsm)
                                          : persist_slots<float>(it.s, c, nsm);
    }
    PF_CUDA(cudaStreamSynchronize(st));
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = res;
  }
  *out = res;
  return PF_OK;
}

size_t filter_sweep_table_bytes(int n) { return (size_t)n * sizeof(BatchItemDev); }

}  // namespace pf

using namespace pf;

extern "C" {

pf_status pf_clenshaw_step(const pf_ham* hh, int32_t prec, int32_t s, const void* V, const void* B1, const void* B2,
                           void* out, double a, double alpha, double beta, int32_t use_H, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H) return PF_EINVAL;
  if (use_H) {
    if (prec != PF_F64) return PF_EINVAL;
    return clenshaw_step_raw(H->D, H->row_ptr, H->col, H->val, prec, s, V, B1, B2, out, a, alpha, beta,
                             (cudaStream_t)stream);
  }
  if (!H->has_rescale) return PF_ESTATE;
  return ham_step(H, prec, s, V, B1, B2, out, a, alpha, beta, (cudaStream_t)stream, 0);
}

pf_status pf_filter_apply(const pf_ham* hh, int32_t prec, int32_t s, const void* V, void* W, const double* coeffs,
                          int32_t K, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H || !V || !W || !coeffs || K < 1) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  if (!valid_prec(prec)) return PF_EINVAL;
  if (!valid_s(s)) return PF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t w = prec_bytes(prec);
  DevBuf a0, a1;
  PF_TRY(a0.alloc(H->D * s * w, st));
  PF_TRY(a1.alloc(H->D * s * w, st));
  return filter_apply_raw(H, prec, s, V, W, coeffs, nullptr, K, a0.p, a1.p, st);
}

pf_status pf_filter_apply_cols(const pf_ham* hh, int32_t prec, int32_t s, const void* V, void* W,
                               const double* coeffs, int32_t K, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H || !V || !W || !coeffs || K < 1) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  if (prec != PF_F64 && prec != PF_F32) return PF_EINVAL;
  if (!valid_s(s)) return PF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t w = prec_bytes(prec);
  const size_t n = (size_t)(K + 1) * s;
  DevBuf a0, a1, tab;
  PF_TRY(a0.alloc(H->D * s * w, st));
  PF_TRY(a1.alloc(H->D * s * w, st));
  PF_TRY(tab.alloc(n * w, st));
  if (prec == PF_F64) {
    PF_CUDA(cudaMemcpyAsync(tab.p, coeffs, n * 8, cudaMemcpyHostToDevice, st));
  } else {
    std::vector<float> c32(n);   // pageable: consumed when the copy call returns
    for (size_t i = 0; i < n; ++i) c32[i] = (float)coeffs[i];
    PF_CUDA(cudaMemcpyAsync(tab.p, c32.data(), n * 4, cudaMemcpyHostToDevice, st));
  }
  return filter_apply_raw(H, prec, s, V, W, nullptr, tab.p, K, a0.p, a1.p, st);
}

pf_status pf_filter_apply_batch(const pf_filter_item* items, int32_t n, int32_t prec, int32_t s, int32_t form,
                                pf_stream_t stream) {
  if (n < 0 || (n > 0 && !items)) return PF_EINVAL;
  if (!valid_prec(prec)) return PF_EINVAL;
  if (!valid_s(s)) return PF_EINVAL;
  if (!(form == PF_FORM_AUTO || form == PF_FORM_STEPS || form == PF_FORM_GRAPH || form == 1 || form == 2 ||
        form == 4 || form == 8 || form == 16))
    return PF_EINVAL;
  if (n == 0) return PF_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t w = prec_bytes(prec);
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
  // the device coefficient tables (pairs for PF_DF64); a pageable source is consumed by the
  // time cudaMemcpyAsync returns
  std::vector<double> ch;
  std::vector<FilterItem> v(n);
  for (int j = 0; j < n; ++j) {
    const Ham* H = reinterpret_cast<const Ham*>(items[j].H);
    unsigned char* base = blob.as<unsigned char>();
    ch.resize(items[j].K + 1);
    coeff_table_host(prec, items[j].coeffs, items[j].K + 1, ch.data());
    PF_CUDA(cudaMemcpyAsync(base + coff[j], ch.data(), (size_t)(items[j].K + 1) * 8, cudaMemcpyHostToDevice, st));
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
  if (form == PF_FORM_STEPS) return filter_sweep(v, table.p, table.bytes, th.data(), st, 0, nullptr);
  if (form == PF_FORM_GRAPH) {
    SweepGraph g;
    PF_TRY(filter_sweep(v, table.p, table.bytes, th.data(), st, 0, &g));
    PF_CUDA(cudaStreamSynchronize(st));   // the graph is released on return
    return PF_OK;
  }
  if (form >= 1) return filter_sweep(v, table.p, table.bytes, th.data(), st, form, nullptr);
  // PF_FORM_AUTO: items of one shape form a group; the autotuner picks the group's form
  std::vector<std::pair<std::pair<int64_t, int64_t>, std::vector<FilterItem>>> shapes;
  for (const FilterItem& it : v) {
    const auto key = std::make_pair(it.H->D, it.H->nnz);
    auto p = std::find_if(shapes.begin(), shapes.end(), [&](const auto& x) { return x.first == key; });
    if (p == shapes.end()) {
      shapes.push_back({key, {}});
      p = shapes.end() - 1;
    }
    p->second.push_back(it);
  }
  for (auto& p : shapes) {
    TuneResult tr;
    PF_TRY(tune_item(p.second[0], st, &tr));
    const int f = choose_form(tr, (int)p.second.size(), nullptr);
    if (f == 0 && p.second.size() == 1) {
      const FilterItem& it = p.second[0];
      PF_TRY(filter_apply_raw(it.H, it.prec, it.s, it.V, it.W, it.coeffs_host, nullptr, it.K, it.aux0, it.aux1, st));
      continue;
    }
    std::vector<unsigned char> tp(filter_sweep_table_bytes((int)p.second.size()));
    DevBuf tb;
    PF_TRY(tb.alloc(tp.size(), st));
    PF_TRY(filter_sweep(p.second, tb.p, tb.bytes, tp.data(), st, f, nullptr));
  }
  return PF_OK;
}

pf_status pf_filter_tune(const pf_ham* hh, int32_t prec, int32_t s, int32_t K, int32_t n, int32_t* form,
                         double* step_us, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H || !form || K < 1 || n < 1) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  if (!valid_prec(prec)) return PF_EINVAL;
  if (!valid_s(s)) return PF_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t w = prec_bytes(prec);
  // a zero start block and zero coefficients: the timing does not depend on the values
  DevBuf V, coeffs;
  PF_TRY(V.alloc((size_t)H->D * s * w, st));
  PF_CUDA(cudaMemsetAsync(V.p, 0, V.bytes, st));
  PF_TRY(coeffs.alloc((size_t)(K + 1) * 8, st));
  PF_CUDA(cudaMemsetAsync(coeffs.p, 0, coeffs.bytes, st));
  FilterItem it;
  it.H = H;
  it.prec = prec;
  it.s = s;
  it.V = V.p;
  it.coeffs_dev = coeffs.as<double>();
  it.K = K;
  TuneResult tr;
  PF_TRY(tune_item(it, st, &tr));
  *form = choose_form(tr, n, nullptr);
  if (step_us) {
    step_us[0] = tr.raw_us;
    step_us[1] = tr.sweep_us;
    step_us[2] = tr.sweep_copies;
    for (int k = 0; k < 5; ++k) step_us[3 + k] = tr.persist_us[k];
  }
  return PF_OK;
}

}  // extern "C"
