// Kernel polynomial method for the density of states (paper Sec. 3.3, Eq. dos_kpm, App. B).
//
// mu_n = Tr T_n(H~) is estimated as (1/R) sum_r <r| T_n(H~) |r> over the R columns of a random
// D x R block with independent zero-mean, unit-variance entries: sqrt(12) (u - 1/2), u the
// SplitMix64 uniforms of the start block (entry (i, r) from counter i R + r).  The Chebyshev
// vectors T_n(H~) V come from the fused Clenshaw step (out = 2 H~ T_n - T_{n-1}), and two
// moments per step come from the doubling identities
//     T_{2n} = 2 T_n^2 - 1,   T_{2n+1} = 2 T_{n+1} T_n - T_1:
//     mu_2n = 2 <T_n V, T_n V> / R - mu_0,   mu_{2n+1} = 2 <T_{n+1} V, T_n V> / R - mu_1,
// with <X, Y> the sum over all entries of X .* Y (a deterministic two-stage reduction).
// The density rho_KPM(x) = [mu_0 g_0 + 2 sum mu_n g_n T_n(x)] / (pi sqrt(1 - x^2)) with the
// Jackson kernel g_n, the :maxdos and (:offset, eta) targets (Sec. 5.2) and K from Eq.
// condition_for_K are evaluated on the host from the N moments.
#include "common.cuh"
#include <cmath>
#include <vector>
#include <algorithm>

namespace pf {

__global__ void kpm_scale_kernel(double* x, int64_t n, double a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] *= a;
}

// part[b] = sum over the entries CTA b visits (grid-stride) of X .* Y
__global__ void kpm_dot_partial(const double* __restrict__ X, const double* __restrict__ Y, int64_t n,
                                double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc = fma(X[i], Y[i], acc);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void kpm_dot_final(const double* __restrict__ part, int np, double* out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = acc;
}

static constexpr int kDotBlocks = 592;   // 148 SMs x 4

static pf_status kpm_dot(const double* X, const double* Y, int64_t n, double* part, double* out, cudaStream_t st) {
  kpm_dot_partial<<<kDotBlocks, 256, 0, st>>>(X, Y, n, part);
  PF_LAUNCH_CHECK("kpm_dot_partial");
  kpm_dot_final<<<1, 256, 0, st>>>(part, kDotBlocks, out);
  PF_LAUNCH_CHECK("kpm_dot_final");
  return PF_OK;
}

static pf_status kpm_moments_impl(const Ham* H, int N, int R, uint64_t seed, double* mu, cudaStream_t st) {
  const int64_t n = H->D * (int64_t)R;
  DevBuf A, B, C, part, dots;
  PF_TRY(A.alloc((size_t)n * 8, st));   // V = T_0 V (kept for mu_0, mu_1), then reused
  PF_TRY(B.alloc((size_t)n * 8, st));
  PF_TRY(C.alloc((size_t)n * 8, st));
  PF_TRY(part.alloc(kDotBlocks * 8, st));
  PF_TRY(dots.alloc((size_t)(N + 2) * 8, st));
  double* V = A.as<double>();
  PF_TRY(start_block_raw(H->D, R, seed, V, st));
  kpm_scale_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(V, n, std::sqrt(12.0));
  PF_LAUNCH_CHECK("kpm_scale_kernel");
  double* d = dots.as<double>();
  // T_1 V = H~ V
  double* Tprev = V;
  double* Tcur = B.as<double>();
  PF_TRY(clenshaw_step_raw(H->D, H->row_ptr, H->col, H->val_t, PF_F64, R, V, V, nullptr, Tcur, 0.0, 1.0, 0.0, st));
  PF_TRY(kpm_dot(V, V, n, part.as<double>(), d + 0, st));      // <V, V>
  PF_TRY(kpm_dot(V, Tcur, n, part.as<double>(), d + 1, st));   // <V, T_1 V>
  // dot slots: 2m -> <T_m, T_m>, 2m + 1 -> <T_{m+1}, T_m>, for m >= 1
  double* spare = C.as<double>();
  bool first = true;
  for (int m = 1; 2 * m < N; ++m) {
    PF_TRY(kpm_dot(Tcur, Tcur, n, part.as<double>(), d + 2 * m, st));
    if (2 * m + 1 >= N) break;
    // T_{m+1} = 2 H~ T_m - T_{m-1}; the first time T_{m-1} is V, which must survive, so the
    // result goes to the spare block; later it overwrites T_{m-1} in place
    double* dst = first ? spare : Tprev;
    PF_TRY(clenshaw_step_raw(H->D, H->row_ptr, H->col, H->val_t, PF_F64, R, Tcur, Tcur, Tprev, dst, 0.0, 2.0, 1.0,
                             st));
    first = false;
    PF_TRY(kpm_dot(dst, Tcur, n, part.as<double>(), d + 2 * m + 1, st));
    Tprev = Tcur;
    Tcur = dst;
  }
  std::vector<double> hd(N + 2, 0.0);
  PF_CUDA(cudaMemcpyAsync(hd.data(), d, (size_t)(N + 2) * 8, cudaMemcpyDeviceToHost, st));
  PF_CUDA(cudaStreamSynchronize(st));
  mu[0] = hd[0] / R;
  if (N > 1) mu[1] = hd[1] / R;
  for (int m = 1; 2 * m < N; ++m) {
    mu[2 * m] = 2.0 * hd[2 * m] / R - mu[0];
    if (2 * m + 1 < N) mu[2 * m + 1] = 2.0 * hd[2 * m + 1] / R - mu[1];
  }
  return PF_OK;
}

static double jackson_g(int n, int N) {
  const double a = M_PI / (N + 1);
  return ((N - n + 1) * std::cos(a * n) + std::sin(a * n) / std::tan(a)) / (N + 1);
}

static double kpm_rho(const double* mu, int N, double x) {
  const double t = std::acos(x);
  double s = mu[0] * jackson_g(0, N);
  for (int n = 1; n < N; ++n) s += 2.0 * mu[n] * jackson_g(n, N) * std::cos(n * t);
  return s / (M_PI * std::sqrt(1.0 - x * x));
}

// P_K(x) of the filter centred at lam_t (Eq. transformation, Eq. transformationCoefficients)
static double filter_at(double lam_t, int K, double x) {
  const double tl = std::acos(lam_t), tx = std::acos(std::max(-1.0, std::min(1.0, x)));
  double chi = 0.0, p = 0.0;
  for (int n = 0; n <= K; ++n) {
    const double c = (n == 0 ? 1.0 : 2.0) * std::cos(n * tl);
    chi += c * std::cos(n * tl);
    p += c * std::cos(n * tx);
  }
  return p / chi;
}

}  // namespace pf

using namespace pf;

extern "C" {

pf_status pf_kpm_moments(pf_ham* hh, int32_t N, int32_t R, uint64_t seed, double* mu, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H || !mu || N < 1) return PF_EINVAL;
  if (!(R == 1 || R == 2 || R == 4 || R == 8 || R == 16 || R == 32 || R == 64)) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  return kpm_moments_impl(H, N, R, seed, mu, (cudaStream_t)stream);
}

pf_status pf_kpm_dos(const double* mu, int32_t N, const double* x, int32_t nx, double* rho) {
  if (!mu || N < 1 || nx < 0 || (nx > 0 && (!x || !rho))) return PF_EINVAL;
  for (int i = 0; i < nx; ++i) {
    if (!(x[i] > -1.0 && x[i] < 1.0)) return PF_EINVAL;
    rho[i] = kpm_rho(mu, N, x[i]);
  }
  return PF_OK;
}

pf_status pf_kpm_target(const double* mu, int32_t N, double eta, double* lam_t) {
  if (!mu || N < 1 || !lam_t || !(eta >= -1.0 && eta <= 1.0)) return PF_EINVAL;
  const int npts = 4001;
  const double edge = 0.999;
  double best = -1.0, xm = 0.0;
  for (int i = 0; i < npts; ++i) {
    const double x = -edge + 2.0 * edge * i / (npts - 1);
    const double r = kpm_rho(mu, N, x);
    if (r > best) {
      best = r;
      xm = x;
    }
  }
  *lam_t = eta >= 0 ? xm + eta * (1.0 - xm) : xm + eta * (xm + 1.0);
  return PF_OK;
}

pf_status pf_choose_K_kpm(const double* mu, int32_t N, double lam_t, int32_t nev, int32_t* K) {
  if (!mu || N < 1 || !K || nev < 1 || !(lam_t > -1.0 && lam_t < 1.0)) return PF_EINVAL;
  const double rho = kpm_rho(mu, N, lam_t);
  if (!(rho > 0.0)) return PF_EINVAL;
  const int nev_g = (int)std::ceil(guard_factor(mu[0]) * nev);   // mu_0 estimates D
  const double delta = nev_g / (2.0 * rho);
  const double k0 = 2.655 * std::sqrt(std::max(1.0 - lam_t * lam_t, 0.0)) / delta;
  int lo = std::max(1, (int)(k0 / 2)), hi = std::max(2, (int)std::ceil(2.0 * k0));
  auto edge = [&](int k) { return std::max(filter_at(lam_t, k, lam_t - delta), filter_at(lam_t, k, lam_t + delta)); };
  const double omega = std::sin(2.655) / 2.655;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (edge(mid) > omega) lo = mid;
    else hi = mid;
  }
  *K = hi;
  return PF_OK;
}

}  // extern "C"
