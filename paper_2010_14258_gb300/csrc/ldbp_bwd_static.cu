// ldbp_backward_static: the learned-DBP adjoint for callers that cannot
// allocate device memory.  Its per-block tap sums go to a file-scope device
// array instead of a caller-provided workspace.
#include <cuda.h>

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

// The address is cached per CUDA context, keyed by the driver's unique
// context id: a device reset destroys the primary context, the module is
// loaded again in the next one and the array may move, so a cached address is
// used only while the context it was looked up in is the current one.
struct StaticAddr {
  unsigned long long ctx_id;
  void* addr;
};
static StaticAddr g_static_addr[kStaticMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Id of the context current on this thread (0 if none), through the
// runtime's driver entry points (no link against the driver library).
static int current_ctx_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return fail(LDBP_ECUDA, "driver entry point cuCtxGetCurrent unavailable");
    get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return fail(LDBP_ECUDA, "driver entry point cuCtxGetId unavailable");
    get_id = reinterpret_cast<CtxGetIdFn>(f);
  }
  CUcontext ctx = nullptr;
  *id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS) return fail(LDBP_ECUDA, "cuCtxGetCurrent failed");
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return fail(LDBP_ECUDA, "cuCtxGetId failed");
  return LDBP_OK;
}

// Device address of g_bwd_scratch in the current context.  The host-side
// name of the array is only a stand-in, so the address is looked up with
// cudaGetSymbolAddress (which also makes the device's primary context current
// if none is) on the first call in a context and cached for that context.
static int static_scratch(void** out) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices)
    return fail(LDBP_EUNSUPPORTED, "device %d beyond the %d devices the static scratch supports", dev,
                kStaticMaxDevices);
  std::lock_guard<std::mutex> lk(g_static_mu);
  unsigned long long id = 0;
  if (int rc = current_ctx_id(&id)) return rc;
  if (id == 0 || !g_static_addr[dev].addr || g_static_addr[dev].ctx_id != id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_bwd_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_bwd_scratch)");
    if (int rc = current_ctx_id(&id)) return rc;
    g_static_addr[dev] = StaticAddr{id, p};
  }
  *out = g_static_addr[dev].addr;
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
