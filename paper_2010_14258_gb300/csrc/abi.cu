// C ABI entry points: argument validation, tile planning and kernel dispatch.
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "ldbp_bwd.cuh"
#include "ldbp_fwd.cuh"

namespace ldbp {

__device__ int g_device_status = 0;

static thread_local char t_last_error[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
  va_end(ap);
}

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(t_last_error, sizeof(t_last_error), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(LDBP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int make_tile_plan(long long n, int H, TilePlan* out, int S) {
  const int Hp = H + (H & 1);
  if (2 * Hp > S / 2) return -1;
  const int Lmax = S - 2 * Hp;
  if (Lmax < 2) return -1;
  long long tpw = (n + Lmax - 1) / Lmax;
  long long L = (n + tpw - 1) / tpw;
  L += L & 1;
  if (L > Lmax) return -1;
  out->Hp = Hp;
  out->L = (int)L;
  out->tiles_per_wave = (int)tpw;
  return 0;
}

static bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bbytes && pb < pa + abytes;
}

// Validates taps/lengths/coefficients shared by the forward and adjoint calls.
static int check_model(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                       long long n, int* H, int* kmax) {
  if (!taps || !T || !c) return fail(LDBP_EINVAL, "taps, T and c must be non-NULL");
  if (M < 1 || M > LDBP_MAX_STEPS) return fail(LDBP_EINVAL, "M=%d outside 1..%d", M, LDBP_MAX_STEPS);
  if (taps_stride < 1) return fail(LDBP_EINVAL, "taps_stride=%d < 1", taps_stride);
  *H = 0;
  *kmax = 0;
  for (int i = 0; i < M; ++i) {
    const int t = T[i];
    if (t < 1 || (t % 2) == 0) return fail(LDBP_EINVAL, "T[%d]=%d must be odd and >= 1", i, t);
    const int K = (t - 1) / 2;
    if (K > LDBP_MAX_HALF_TAPS) return fail(LDBP_EINVAL, "T[%d]=%d exceeds the supported length %d", i, t,
                                            2 * LDBP_MAX_HALF_TAPS + 1);
    if (K + 1 > taps_stride) return fail(LDBP_EINVAL, "T[%d]=%d needs taps_stride >= %d", i, t, K + 1);
    if (!std::isfinite(c[i])) return fail(LDBP_ENONFINITE, "c[%d] is NaN or infinite", i);
    *H += K;
    *kmax = K > *kmax ? K : *kmax;
  }
  (void)n;
  return 0;
}

// One mbarrier expecting two arrivals, `arrivals` of them made, then the
// library's bounded wait on the phase (see ldbp_wait_probe).
__global__ void wait_probe_kernel(int arrivals, int limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x < arrivals) mbar_arrive(&bar);
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, limit);
}

}  // namespace ldbp

using namespace ldbp;

extern "C" {

int ldbp_wait_probe(int32_t arrivals, int32_t limit, void* stream) {
  if (arrivals < 0 || arrivals > 2) return fail(LDBP_EINVAL, "arrivals=%d outside 0..2", arrivals);
  if (limit < 1 || limit > (1 << 20)) return fail(LDBP_EINVAL, "limit=%d outside 1..2^20", limit);
  wait_probe_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(arrivals, limit);
  LDBP_CUDA_TRY(cudaGetLastError());
  return LDBP_OK;
}

const char* ldbp_last_error(void) { return t_last_error; }

int ldbp_version(void) { return 100; }

int ldbp_device_status(void) {
  int h = 0;
  LDBP_CUDA_TRY(cudaDeviceSynchronize());
  LDBP_CUDA_TRY(cudaMemcpyFromSymbol(&h, g_device_status, sizeof(int)));
  const int zero = 0;
  LDBP_CUDA_TRY(cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int)));
  if (h == kDevTimeout) return fail(LDBP_ETIMEOUT, "a bounded device wait ran out");
  if (h != 0) return fail(LDBP_ECUDA, "device status %d", h);
  return LDBP_OK;
}

int ldbp_apply(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M, const void* x,
               void* y, int64_t n, int32_t batch, void* ckpt, void* stream) {
  if (!x || !y) return fail(LDBP_EINVAL, "x and y must be non-NULL");
  if (n < 1 || batch < 1) return fail(LDBP_EINVAL, "n=%lld, batch=%d must be >= 1", (long long)n, batch);
  int H = 0, kmax = 0;
  if (int rc = check_model(taps, taps_stride, T, c, M, n, &H, &kmax)) return rc;
  const size_t bytes = (size_t)n * (size_t)batch * sizeof(float2);
  if (overlaps(x, bytes, y, bytes)) return fail(LDBP_EINVAL, "x and y overlap");
  if (ckpt && (overlaps(ckpt, bytes * M, x, bytes) || overlaps(ckpt, bytes * M, y, bytes)))
    return fail(LDBP_EINVAL, "ckpt overlaps x or y");
  int Ks[LDBP_MAX_STEPS];
  for (int i = 0; i < M; ++i) Ks[i] = (T[i] - 1) / 2;
  TilePlan plan;
  if (make_tile_plan(n, H, &plan, fwd_tile_samples(Ks, M, kmax)))
    return fail(LDBP_EINVAL, "halo sum %d too large for one tile", H);
  if ((long long)plan.tiles_per_wave * batch > 0x7fffffffLL) return fail(LDBP_EINVAL, "grid too large");
  FwdParams p;
  memset(&p, 0, sizeof(p));
  p.x = static_cast<const float2*>(x);
  p.y = static_cast<float2*>(y);
  p.ckpt = static_cast<float2*>(ckpt);
  p.taps = static_cast<const float2*>(taps);
  p.taps_stride = taps_stride;
  p.n = n;
  p.batch = batch;
  p.M = M;
  p.tiles_per_wave = plan.tiles_per_wave;
  p.L = plan.L;
  p.Hp = plan.Hp;
  for (int i = 0; i < M; ++i) {
    p.K[i] = (T[i] - 1) / 2;
    p.c[i] = c[i];
  }
  cudaError_t e = launch_ldbp_fwd(p, kmax, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "ldbp_fwd launch");
  return LDBP_OK;
}

}  // extern "C"

namespace ldbp {

// Backward tile plan: halo H + K_max per side (see ldbp_bwd.cu).
static int bwd_plan(long long n, const int32_t* T, int M, TilePlan* plan, int* kmax) {
  int H = 0;
  *kmax = 0;
  for (int i = 0; i < M; ++i) {
    const int K = (T[i] - 1) / 2;
    H += K;
    *kmax = K > *kmax ? K : *kmax;
  }
  return make_tile_plan(n, H + *kmax, plan);
}

}  // namespace ldbp

extern "C" {

int ldbp_backward_workspace(int64_t n, int32_t batch, const int32_t* T, int32_t M, size_t* bytes) {
  if (!T || !bytes) return fail(LDBP_EINVAL, "T and bytes must be non-NULL");
  if (M < 1 || M > LDBP_MAX_STEPS) return fail(LDBP_EINVAL, "M=%d outside 1..%d", M, LDBP_MAX_STEPS);
  if (n < 1 || batch < 1) return fail(LDBP_EINVAL, "n=%lld, batch=%d must be >= 1", (long long)n, batch);
  for (int i = 0; i < M; ++i)
    if (T[i] < 1 || T[i] % 2 == 0 || (T[i] - 1) / 2 > LDBP_MAX_HALF_TAPS)
      return fail(LDBP_EINVAL, "T[%d]=%d must be odd in 1..%d", i, T[i], 2 * LDBP_MAX_HALF_TAPS + 1);
  TilePlan plan;
  int kmax = 0;
  if (bwd_plan(n, T, M, &plan, &kmax)) return fail(LDBP_EINVAL, "halo sum too large for one tile");
  const int cls = fwd_kmax_class(kmax);
  *bytes = (size_t)plan.tiles_per_wave * (size_t)batch * (size_t)M * (size_t)(cls + 2) * sizeof(float2);
  return LDBP_OK;
}

int ldbp_backward(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                  const void* ckpt, const void* gy, void* gx, void* gtaps, int64_t n, int32_t batch, void* workspace,
                  size_t workspace_bytes, void* stream) {
  return ldbp_backward_c(taps, taps_stride, T, c, M, ckpt, gy, gx, gtaps, nullptr, n, batch, workspace,
                         workspace_bytes, stream);
}

int ldbp_backward_c(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, int32_t M,
                    const void* ckpt, const void* gy, void* gx, void* gtaps, float* gc, int64_t n, int32_t batch,
                    void* workspace, size_t workspace_bytes, void* stream) {
  if (!ckpt || !gy || !gtaps || !workspace)
    return fail(LDBP_EINVAL, "ckpt, gy, gtaps and workspace must be non-NULL");
  if (n < 1 || batch < 1) return fail(LDBP_EINVAL, "n=%lld, batch=%d must be >= 1", (long long)n, batch);
  int H = 0, kmax = 0;
  if (int rc = check_model(taps, taps_stride, T, c, M, n, &H, &kmax)) return rc;
  size_t need = 0;
  if (int rc = ldbp_backward_workspace(n, batch, T, M, &need)) return rc;
  if (workspace_bytes < need)
    return fail(LDBP_EINVAL, "workspace of %zu bytes is smaller than the %zu bytes needed", workspace_bytes, need);
  const size_t bytes = (size_t)n * (size_t)batch * sizeof(float2);
  if (gx && (overlaps(gx, bytes, gy, bytes) || overlaps(gx, bytes, ckpt, bytes * M)))
    return fail(LDBP_EINVAL, "gx overlaps gy or ckpt");
  TilePlan plan;
  bwd_plan(n, T, M, &plan, &kmax);
  if ((long long)plan.tiles_per_wave * batch > 0x7fffffffLL) return fail(LDBP_EINVAL, "grid too large");
  const int cls = fwd_kmax_class(kmax);
  BwdParams p;
  memset(&p, 0, sizeof(p));
  p.ckpt = static_cast<const float2*>(ckpt);
  p.gy = static_cast<const float2*>(gy);
  p.gx = static_cast<float2*>(gx);
  p.partial = static_cast<float2*>(workspace);
  p.taps = static_cast<const float2*>(taps);
  p.taps_stride = taps_stride;
  p.n = n;
  p.batch = batch;
  p.M = M;
  p.tiles_per_wave = plan.tiles_per_wave;
  p.L = plan.L;
  p.Hp = plan.Hp;
  TapReduceK kk;
  memset(&kk, 0, sizeof(kk));
  for (int i = 0; i < M; ++i) {
    p.K[i] = (T[i] - 1) / 2;
    p.c[i] = c[i];
    kk.K[i] = p.K[i];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_ldbp_bwd(p, cls, st);
  if (e != cudaSuccess) return cuda_fail(e, "ldbp_bwd launch");
  e = launch_tap_reduce(p.partial, plan.tiles_per_wave * batch, M, cls + 2, kk, static_cast<float2*>(gtaps),
                        taps_stride, st);
  if (e != cudaSuccess) return cuda_fail(e, "tap reduce launch");
  if (gc) {
    e = launch_c_reduce(p.partial, plan.tiles_per_wave * batch, M, cls + 2, gc, st);
    if (e != cudaSuccess) return cuda_fail(e, "c reduce launch");
  }
  return LDBP_OK;
}

}  // extern "C"
