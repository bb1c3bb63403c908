// Optimiser step of learned-DBP training (Sec. IV-B: Adam) with the pruning
// mask of Sec. IV-C: taps beyond the current half-width K_i are held at zero.
#include <cmath>

#include "common.cuh"

namespace ldbp {

struct AdamK {
  int K[LDBP_MAX_STEPS];
};

// Adam on the real and imaginary parts of every tap (bias-corrected moments).
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int M, int stride, const __grid_constant__ AdamK kk, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // real index over [M][stride][2]
  if (e >= M * stride * 2) return;
  const int i = e / (2 * stride), k = (e / 2) - i * stride;
  if (k > kk.K[i]) {  // pruned (or unused) tap: masked to zero
    theta[e] = 0.f;
    m[e] = 0.f;
    v[e] = 0.f;
    return;
  }
  const float gg = g[e];
  const float mm = b1 * m[e] + (1.f - b1) * gg;
  const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
  m[e] = mm;
  v[e] = vv;
  theta[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

}  // namespace ldbp

using namespace ldbp;

extern "C" int ldbp_adam_step(void* taps, const void* gtaps, float* m, float* v, const int32_t* T, int32_t M,
                              int32_t taps_stride, int32_t step, float lr, float beta1, float beta2, float eps,
                              void* stream) {
  if (!taps || !gtaps || !m || !v || !T) return fail(LDBP_EINVAL, "taps, gtaps, m, v and T must be non-NULL");
  if (M < 1 || M > LDBP_MAX_STEPS || taps_stride < 1) return fail(LDBP_EINVAL, "bad M or taps_stride");
  if (step < 1) return fail(LDBP_EINVAL, "step counts from 1");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return fail(LDBP_EINVAL, "bad Adam hyper-parameters");
  AdamK kk;
  for (int i = 0; i < LDBP_MAX_STEPS; ++i) kk.K[i] = 0;
  for (int i = 0; i < M; ++i) {
    if (T[i] < 1 || T[i] % 2 == 0 || (T[i] - 1) / 2 + 1 > taps_stride)
      return fail(LDBP_EINVAL, "T[%d]=%d must be odd with (T-1)/2 < taps_stride", i, T[i]);
    kk.K[i] = (T[i] - 1) / 2;
  }
  const double c1 = 1.0 - std::pow((double)beta1, (double)step), c2 = 1.0 - std::pow((double)beta2, (double)step);
  const int total = M * taps_stride * 2;
  adam_kernel<<<(total + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<float*>(taps), static_cast<const float*>(gtaps), m, v, M, taps_stride, kk, lr, beta1, beta2, eps,
      (float)c1, (float)c2);
  LDBP_CUDA_TRY(cudaGetLastError());
  return LDBP_OK;
}
