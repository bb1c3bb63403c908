// Microbenchmarks that measure the arithmetic ceilings the roofline of the
// fused kernels is quoted against: scalar FP32 FMA, packed FP32x2 FMA and
// special-function (sin) throughput, on every SM of the current device.
#include <cuda_runtime.h>

#include "common.cuh"

namespace ldbp {

constexpr int kUbChains = 8;

__global__ void __launch_bounds__(256) ub_ffma(float* out, int iters, float a, float b) {
  float x[kUbChains];
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) x[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kUbChains; ++k) x[k] = fmaf(x[k], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) s += x[k];
  if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ub_ffma2(float* out, int iters, float a, float b) {
  float2 x[kUbChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) x[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kUbChains; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) s += x[k].x + x[k].y;
  if (s == 1234.5f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ub_sin(float* out, int iters, float a, float b) {
  float x[kUbChains];
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) x[k] = threadIdx.x * 1e-3f + k * 0.1f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kUbChains; ++k) x[k] = __sinf(x[k]);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) s += x[k];
  if (s == 1234.5f) out[threadIdx.x] = s + a + b;
}

// Packed and scalar FMAs interleaved (independent chains): shows whether the
// two FMA pipes of an SM sub-partition can run both instruction kinds at once.
__global__ void __launch_bounds__(256) ub_mixed(float* out, int iters, float a, float b) {
  float2 x[kUbChains / 2];
  float y[kUbChains];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int k = 0; k < kUbChains / 2; ++k) x[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f);
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) y[k] = threadIdx.x * 2e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < kUbChains / 2; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
#pragma unroll
      for (int k = 0; k < kUbChains; ++k) y[k] = fmaf(y[k], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kUbChains / 2; ++k) s += x[k].x + x[k].y;
#pragma unroll
  for (int k = 0; k < kUbChains; ++k) s += y[k];
  if (s == 1234.5f) out[threadIdx.x] = s;
}

}  // namespace ldbp

using namespace ldbp;

extern "C" int ldbp_ubench(int32_t kind, double* ops_per_second) {
  if (!ops_per_second) return fail(LDBP_EINVAL, "ops_per_second must be non-NULL");
  if (kind < 0 || kind > 3) return fail(LDBP_EINVAL, "kind=%d outside 0..3", kind);
  int dev = 0, sms = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  LDBP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  float* out = nullptr;
  LDBP_CUDA_TRY(cudaMalloc(&out, 256 * sizeof(float)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  const int iters = kind == 2 ? 4096 : 16384;
  auto launch = [&](int it) {
    if (kind == 0) ub_ffma<<<blocks, threads>>>(out, it, 0.999f, 1e-3f);
    else if (kind == 1) ub_ffma2<<<blocks, threads>>>(out, it, 0.999f, 1e-3f);
    else if (kind == 2) ub_sin<<<blocks, threads>>>(out, it, 0.f, 0.f);
    else ub_mixed<<<blocks, threads>>>(out, it, 0.999f, 1e-3f);
  };
  launch(64);  // warm-up
  cudaEventRecord(e0);
  launch(iters);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return cuda_fail(err, "ubench");
  const double per_iter = kind == 1 ? 2.0 * kUbChains : kind == 3 ? 2.0 * kUbChains : (double)kUbChains;
  const double lane_ops = (double)blocks * threads * iters * 4.0 * per_iter;
  *ops_per_second = lane_ops / (ms * 1e-3);
  return LDBP_OK;
}
