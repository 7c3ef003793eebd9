// block_inner_noalloc: the Gram product G = X^dagger Y for callers that are
// not allowed to allocate device memory.
//
// block_inner keeps its per-CTA partial Gram matrices in a workspace that the
// library allocates (and grows) with cudaMalloc on first use.  Some callers
// cannot accept that: a host application whose device memory is entirely
// owned by another framework's pool or capped by its scheduler, or a
// latency-critical loop in which a cudaMalloc (which can synchronise the
// device, and can fail under memory pressure halfway through a solve) is not
// permitted.  This entry point computes the same product with the same
// kernels, but its partials live in a fixed array compiled into the library,
// so the call itself allocates nothing.
//
// The array is kStaticSlots complex128 values (2 MiB); every GPU that loads
// the library holds it until the process exits.  With CUDA's lazy module
// loading (the default) the array is created when the library's device code
// is first loaded on a device, which the first call here triggers through
// cudaGetSymbolAddress: that first call on each device may therefore take
// device memory (and can fail if none is left), later calls take none.  A
// caller that must not allocate inside its loop makes one call at set-up
// (N = 0 is enough), with the device current and before any stream capture.
// All calls on a device share the array: calls whose kernels overlap on the
// GPU (for example issued on two streams without ordering) race on it and
// give wrong results.  Each call writes every partial it later reads, so no
// state carries over from the previous call and nothing needs clearing.
// The device address is cached per device for the life of the process; the
// library (this entry point, and every operator) must not be used across a
// cudaDeviceReset, after which the cached address is no longer valid.
#include <mutex>

#include "internal.cuh"

namespace mrhs {
namespace {

constexpr int64_t kStaticSlots = 131072;   // complex128 partial-Gram entries (2 MiB)

static __device__ __align__(256) double2 g_noalloc_partials[kStaticSlots];

// Host code must not use g_noalloc_partials directly (on the host it names a
// stand-in, not device memory): the device address is looked up once per
// device, with that device current, and cached here.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double2* g_dev_ptr[kMaxDevices] = {nullptr};

int partials_for_current_device(double2** out) {
  int dev = 0;
  MRHS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MRHS_ERR_INVALID_ARG, "device ordinal too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
      return fail(MRHS_ERR_CUDA, std::string("cudaGetSymbolAddress(static Gram scratch): ") +
                                     cudaGetErrorString(e));
    g_dev_ptr[dev] = (double2*)p;
  }
  *out = g_dev_ptr[dev];
  return MRHS_OK;
}

}  // namespace
}  // namespace mrhs

using namespace mrhs;

extern "C" int block_inner_noalloc(const void* X, const void* Y, void* G, int64_t N, int32_t rx,
                                   int32_t ry, int32_t dtype, void* stream) {
  if (N < 0) return fail(MRHS_ERR_INVALID_ARG, "block_inner_noalloc: N < 0");
  if (rx < 1 || ry < 1 || rx > MRHS_MAX_RHS || ry > MRHS_MAX_RHS)
    return fail(MRHS_ERR_INVALID_ARG,
                "block_inner_noalloc: rx and ry must be in 1..64 (the static scratch holds "
                "partial Gram matrices of at most 64 x 64)");
  if (dtype != MRHS_C128 && dtype != MRHS_C64)
    return fail(MRHS_ERR_INVALID_ARG, "block_inner_noalloc: dtype");
  if (!G || ((uintptr_t)G & 15u)) return fail(MRHS_ERR_INVALID_ARG, "G null or misaligned");
  if (N > 0 && (!X || !Y || ((uintptr_t)X & 15u) || ((uintptr_t)Y & 15u)))
    return fail(MRHS_ERR_INVALID_ARG, "X or Y null or misaligned");
  double2* part = nullptr;
  MRHS_TRY(partials_for_current_device(&part));
  return gram_ws_capped(X, Y, (double2*)G, N, rx, ry, dtype, part, kStaticSlots,
                        (cudaStream_t)stream);
}
