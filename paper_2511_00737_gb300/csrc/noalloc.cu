// bfv_ptct_similarity_noalloc: the encrypted-similarity stage with its scratch in a
// fixed device array compiled into the library, for callers that cannot allocate
// device memory at run time (see include/ephdc.h).  It launches the same kernels as
// bfv_ptct_similarity; only the location of the scratch differs.
#include <cstdio>

#include "ephdc_internal.cuh"

// The scratch: split partial sums, two score-accumulator buffers and the key-switch
// digits.  Held by every device that loads the library, for the life of the process.
static __device__ __align__(256) uint32_t g_static_scratch[EPHDC_STATIC_SCRATCH_BYTES / 4];

namespace {

constexpr int kMaxDevices = 256;

// Device address of g_static_scratch on the current device.  In host code the symbol
// only names a host-side stand-in, so kernels must be given this address, never
// &g_static_scratch.  Looked up on every call (a host-side query), so that it stays
// valid when the module is loaded anew after a cudaDeviceReset.
cudaError_t scratch_address(uint32_t** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<uint32_t*>(p);
  return cudaSuccess;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" ephdc_status bfv_ptct_similarity_noalloc(ephdc_ctx* ctx, const uint32_t* pt, int32_t B,
                                                    const void* model, const void* gk,
                                                    uint32_t* out, void* stream) {
  if (!ctx) return EPHDC_EINVAL;
  ephdc::ctx_clear_error(ctx);
  const DevCtx& d = *ephdc::ctx_dev(ctx);
  if (!pt || !model || !out || (d.logr && !gk))
    return ephdc::ctx_fail(ctx, EPHDC_EINVAL, "a required device pointer is NULL");
  if (!aligned16(pt) || !aligned16(model) || !aligned16(out) || (gk && !aligned16(gk)))
    return ephdc::ctx_fail(ctx, EPHDC_EINVAL, "device pointers must be 16-byte aligned");
  if (B < 1) return ephdc::ctx_fail(ctx, EPHDC_EINVAL, "batch must be positive");
  if (d.layout || d.compact || d.mdig)
    return ephdc::ctx_fail(ctx, EPHDC_EUNSUPPORTED,
                           "the static-scratch path needs layout 0 and the full residue model");

  const size_t G = ((size_t)B + d.cap - 1) / d.cap;
  const size_t count = G * d.Kp;
  const size_t acc_words = count * 2 * d.L * d.n;   // one set of score accumulators
  const size_t dig_words = count * d.L * d.n;       // key-switch digits
  const size_t cap_words = EPHDC_STATIC_SCRATCH_BYTES / 4;
  const size_t fixed = 2 * acc_words + dig_words;
  if (fixed + acc_words > cap_words) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "batch of %d needs %zu bytes of scratch; the static scratch holds %u bytes "
             "(use bfv_ptct_similarity for this size)",
             (int)B, (fixed + acc_words) * 4, EPHDC_STATIC_SCRATCH_BYTES);
    return ephdc::ctx_fail(ctx, EPHDC_EINVAL, msg);
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return ephdc::ctx_fail(ctx, EPHDC_ECUDA, "no current CUDA device");
  if (dev != ephdc::ctx_device(ctx))
    return ephdc::ctx_fail(ctx, EPHDC_EINVAL, "the current device is not the context's device");
  uint32_t* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return ephdc::ctx_fail(ctx, EPHDC_ECUDA, cudaGetErrorString(e));

  // layout: acc | tmp | digits | partial sums (as many splits as fit)
  uint32_t* acc = base;
  uint32_t* tmp = acc + acc_words;
  uint32_t* digits = tmp + acc_words;
  uint32_t* partial = digits + dig_words;
  const int splits_fit = (int)((cap_words - fixed) / acc_words);
  cudaStream_t st = (cudaStream_t)stream;

  e = ephdc::launch_mac(d, pt, (int)G, (const uint32_t*)model, partial, splits_fit, acc, st);
  if (e == cudaSuccess && d.logr)
    e = ephdc::launch_rotate_sum(d, acc, tmp, digits, (int)count, (const uint32_t*)gk, st);
  const uint32_t* cur = (d.logr & 1) ? tmp : acc;  // ping-pong ends in tmp after odd steps
  if (e == cudaSuccess) e = ephdc::launch_export(d, cur, (int)count, out, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return ephdc::ctx_fail(ctx, EPHDC_ECUDA, cudaGetErrorString(e));
  return EPHDC_OK;
}
