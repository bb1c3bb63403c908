// ldbp_backward_static: the learned-DBP adjoint for callers that cannot
// allocate device memory.  Its per-block tap sums go to a file-scope device
// array instead of a caller-provided workspace.
#include <mutex>

#include "common.cuh"
#include "ldbp_bwd.cuh"

namespace ldbp {

constexpr size_t kStaticScratchBytes = LDBP_STATIC_SCRATCH_BYTES;
constexpr int kStaticMaxDevices = 64;

// Loaded with the library's device code: every GPU that loads the library
// holds these bytes until the process exits.
static __device__ __align__(256) float2 g_bwd_scratch[kStaticScratchBytes / sizeof(float2)];

static std::mutex g_static_mu;
static void* g_static_addr[kStaticMaxDevices] = {};

// Device address of g_bwd_scratch on the current device.  The host-side name
// of the array is only a stand-in, so the address is looked up once per
// device (with that device current) and cached.
static int static_scratch(void** out) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices)
    return fail(LDBP_EUNSUPPORTED, "device %d beyond the %d devices the static scratch supports", dev,
                kStaticMaxDevices);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_bwd_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_bwd_scratch)");
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return LDBP_OK;
}

}  // namespace ldbp

using namespace ldbp;

extern "C" int ldbp_backward_static(const void* taps, int32_t taps_stride, const int32_t* T, const float* c,
                                    int32_t M, const void* ckpt, const void* gy, void* gx, void* gtaps, int64_t n,
                                    int32_t batch, void* stream) {
  size_t need = 0;
  if (int rc = ldbp_backward_workspace(n, batch, T, M, &need)) return rc;
  if (need > kStaticScratchBytes)
    return fail(LDBP_EINVAL,
                "ldbp_backward_static needs %zu bytes of scratch for this problem but its static array holds %zu "
                "(LDBP_STATIC_SCRATCH_BYTES); use ldbp_backward with a caller workspace",
                need, kStaticScratchBytes);
  void* ws = nullptr;
  if (int rc = static_scratch(&ws)) return rc;
  return ldbp_backward(taps, taps_stride, T, c, M, ckpt, gy, gx, gtaps, n, batch, ws, kStaticScratchBytes, stream);
}
