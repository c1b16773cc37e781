// Pair-float arithmetic shared by the Clenshaw steps and the tall-skinny dense kernels.
#pragma once
#include <cuda_runtime.h>

namespace pf {

// ------------------------------------------------------------------ pair-float arithmetic
// A value held as the unevaluated sum hi + lo of two floats (Dekker 1971; on GPUs, Thall 2006).
// The step needs x * y + z only, built from two error-free transformations:
//   two_prod: x y = p + e exactly, p = rn(x y), e = fma(x, y, -p);
//   two_sum (Knuth): a + b = s + t exactly, s = rn(a + b), w = rn(s - a),
//                    t = rn(rn(a - rn(s - w)) + rn(b - w)).
// x * y + z keeps hi = two_sum(z.hi, p).s and lo = z.lo + (t + e + x.hi y.lo + x.lo y.hi)
// (x.lo y.lo, below 2^-48 of the product, is dropped), so a chain of them is the compensated
// dot product of Ogita, Rump and Oishi (2005): error about 2^-47 relative to the sum of the
// terms' magnitudes.  Results stay unnormalised (|lo| may exceed half an ulp of hi) until a
// step stores them.  Every operation is an _rn intrinsic, which the compiler neither
// contracts into an FMA nor reorders: the transformations are exact only as written.
struct __align__(8) df2 {
  float hi, lo;
  df2() = default;
  __host__ __device__ constexpr df2(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit constexpr df2(int x) : hi((float)x), lo(0.0f) {}
  __host__ __device__ explicit df2(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

__host__ __device__ __forceinline__ df2 operator-(df2 a) { return df2(-a.hi, -a.lo); }
__host__ __device__ __forceinline__ bool operator!=(df2 a, df2 b) { return a.hi != b.hi || a.lo != b.lo; }
__device__ __forceinline__ df2 operator*(df2 x, df2 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df2(p, e);
}
__device__ __forceinline__ df2 df_fma(df2 x, df2 y, df2 z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const float s = __fadd_rn(z.hi, p);
  const float w = __fsub_rn(s, z.hi);
  const float t = __fadd_rn(__fsub_rn(z.hi, __fsub_rn(s, w)), __fsub_rn(p, w));
  return df2(s, __fadd_rn(z.lo, __fadd_rn(t, e)));
}
// two_sum(hi, lo): the stored form, |lo| <= half an ulp of hi
__device__ __forceinline__ df2 df_norm(df2 a) {
  const float s = __fadd_rn(a.hi, a.lo);
  const float w = __fsub_rn(s, a.hi);
  return df2(s, __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, w)), __fsub_rn(a.lo, w)));
}

}  // namespace pf
