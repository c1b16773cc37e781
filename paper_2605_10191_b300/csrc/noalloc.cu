// Allocation-free variant of the K-step filter application (pf_filter_apply).
//
// pf_filter_apply needs two D x s auxiliary blocks for the Clenshaw recurrence and gets
// them from the library's allocator on every call.  Some callers cannot allow that: code
// running while a memory pool is frozen or exhausted, hosts whose allocator must not be
// re-entered from inside their own hooks, or real-time loops that forbid allocation calls.
// pf_filter_apply_noalloc takes the two blocks from one fixed device array instead, so it
// calls no allocation routine at all.
#include "common.cuh"

namespace pf {

// Fixed scratch shared by every call of pf_filter_apply_noalloc: room for both auxiliary
// blocks (each rounded up to 256 bytes).  Every device that loads the library holds it
// until the process exits.
#define PF_NOALLOC_SCRATCH_BYTES (32ull << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[PF_NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side shadow, not device memory.  The device
// address is looked up on every call, with the caller's device current: the query allocates
// nothing, costs far less than the K steps it precedes, and after cudaDeviceReset (or anything
// else that destroys and re-creates the primary context, which reloads the module and can move
// the array) the next call gets the new address instead of a stale one.
static pf_status noalloc_scratch_address(void** out) {
  void* p = nullptr;
  PF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  if (!p) return PF_ECUDA;
  *out = p;
  return PF_OK;
}

}  // namespace pf

using namespace pf;

extern "C" pf_status pf_filter_apply_noalloc(const pf_ham* hh, int32_t prec, int32_t s, const void* V, void* W,
                                             const double* coeffs, int32_t K, pf_stream_t stream) {
  const Ham* H = reinterpret_cast<const Ham*>(hh);
  if (!H || !V || !W || !coeffs || K < 1) return PF_EINVAL;
  if (!H->has_rescale) return PF_ESTATE;
  if (!valid_prec(prec)) return PF_EINVAL;
  if (!(s == 1 || s == 2 || s == 4 || s == 8 || s == 16 || s == 32 || s == 64)) return PF_EINVAL;
  const size_t w = prec_bytes(prec);
  const size_t blk = ((size_t)H->D * (size_t)s * w + 255) & ~(size_t)255;
  if (2 * blk > PF_NOALLOC_SCRATCH_BYTES) return PF_EINVAL;   // too large for the fixed scratch
  void* base = nullptr;
  PF_TRY(noalloc_scratch_address(&base));
  // The recurrence never reads the auxiliary blocks before writing them (b_{K+1} and
  // b_{K+2} are zero and are skipped), so the previous call's contents need no clearing.
  void* aux0 = base;
  void* aux1 = static_cast<unsigned char*>(base) + blk;
  return filter_apply_raw(H, prec, s, V, W, coeffs, nullptr, K, aux0, aux1, (cudaStream_t)stream);
}
