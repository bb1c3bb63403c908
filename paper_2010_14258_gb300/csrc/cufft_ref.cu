// Library-FFT split-step (cuFFT + elementwise kernels), the comparison path
// for the fused cluster-resident kernel.  Runs the same FP64-built programs
// step by step: forward FFT, spectral multiply (+ ASE), inverse FFT, Kerr.
// cuFFT takes any length, so this path also simulates the non-power-of-two
// grids of the analog-rate channel (e.g. 6 samples/symbol).
#include <cufft.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <string>

#include "common.cuh"
#include "cufft_plan.cuh"
#include "philox.cuh"
#include "ssm_host.cuh"

namespace ldbp {

__global__ void spectral_kernel(float2* __restrict__ X, const float2* __restrict__ tab,
                                const uint32_t* __restrict__ tab_lo, float lo_scale, float scale,
                                const float2* __restrict__ ntab, int noise, float noise_std, float flat, int span,
                                uint32_t counter, uint32_t seed_lo, uint32_t seed_hi, long long n, long long total) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total;
       m += (long long)gridDim.x * blockDim.x) {
    const long long b = m / n, k = m - b * n;
    float2 A = cmul_hl(X[m], tab[k], tail_h2(tab_lo[k], lo_scale));
    A = make_float2(A.x * scale, A.y * scale);
    if (noise) {
      const float2 g = ase_normal((uint32_t)k, (uint32_t)b, (uint32_t)span, counter, seed_lo, seed_hi);
      const float2 hn = ntab ? ntab[k] : make_float2(flat, 0.f);
      A = cadd(A, cmul(hn, make_float2(g.x * noise_std, g.y * noise_std)));
    }
    X[m] = A;
  }
}

__global__ void kerr_kernel(float2* __restrict__ x, float c, long long total) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total;
       m += (long long)gridDim.x * blockDim.x)
    x[m] = kerr_rotate_precise<true>(x[m], c);
}

static std::mutex g_plan_mu;
static std::map<std::string, cufftHandle> g_plans;

int cufft_plan(long long n, int batch, cudaStream_t st, cufftHandle* out) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  char key[96];
  snprintf(key, sizeof(key), "%d:%p:%lld:%d", dev, (void*)st, n, batch);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find(key);
  if (it == g_plans.end()) {
    cufftHandle h;
    long long nn = n;
    size_t ws = 0;
    if (cufftCreate(&h) != CUFFT_SUCCESS) return fail(LDBP_ECUDA, "cufftCreate failed");
    if (cufftMakePlanMany64(h, 1, &nn, nullptr, 1, n, nullptr, 1, n, CUFFT_C2C, batch, &ws) != CUFFT_SUCCESS) {
      cufftDestroy(h);
      return fail(LDBP_ECUDA, "cufftMakePlanMany64 failed for n=%lld batch=%d", n, batch);
    }
    if (cufftSetStream(h, st) != CUFFT_SUCCESS) {
      cufftDestroy(h);
      return fail(LDBP_ECUDA, "cufftSetStream failed");
    }
    it = g_plans.emplace(key, h).first;
  }
  *out = it->second;
  return 0;
}

}  // namespace ldbp

using namespace ldbp;

extern "C" int ssm_cufft(const ldbp_fiber* fiber, const ldbp_link* link, double fs_hz, int32_t dbp_steps_per_span,
                         int32_t dbp_symmetric, const void* x, void* y, int64_t n, int32_t batch, void* stream) {
  if (int rc = check_link(fiber, link, fs_hz, x, y, n, batch, /*pow2=*/false)) return rc;
  if (dbp_steps_per_span < 0) return fail(LDBP_EINVAL, "dbp_steps_per_span must be >= 0");
  std::shared_ptr<DeviceProgram> dp;
  if (int rc = link_program(*fiber, *link, fs_hz, n, dbp_steps_per_span, dbp_symmetric != 0, &dp)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cufftHandle plan;
  if (int rc = cufft_plan(n, batch, st, &plan)) return rc;
  const long long total = n * (long long)batch;
  float2* Y = static_cast<float2*>(y);
  if (x != y) LDBP_CUDA_TRY(cudaMemcpyAsync(y, x, total * sizeof(float2), cudaMemcpyDeviceToDevice, st));
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  if (dp->c_pre != 0.f) kerr_kernel<<<blocks, 256, 0, st>>>(Y, dp->c_pre, total);
  const uint64_t seed = dbp_steps_per_span ? 0 : link->seed, ctr = dbp_steps_per_span ? 0 : link->counter;
  for (const SsmStep& s : dp->host_steps) {
    if (cufftExecC2C(plan, (cufftComplex*)Y, (cufftComplex*)Y, CUFFT_FORWARD) != CUFFT_SUCCESS)
      return fail(LDBP_ECUDA, "cufftExecC2C forward failed");
    spectral_kernel<<<blocks, 256, 0, st>>>(Y, dp->tabs[s.tab], dp->tabs_lo[s.tab], dp->tabs_lo_scale[s.tab], s.scale,
                                            s.noise_tab >= 0 ? dp->tabs[s.noise_tab] : nullptr,
                                            s.noise_tab > -2, dp->noise_std, 1.0f / (float)n, s.span,
                                            (uint32_t)ctr, (uint32_t)seed, (uint32_t)(seed >> 32), n, total);
    if (cufftExecC2C(plan, (cufftComplex*)Y, (cufftComplex*)Y, CUFFT_INVERSE) != CUFFT_SUCCESS)
      return fail(LDBP_ECUDA, "cufftExecC2C inverse failed");
    if (s.c != 0.f) kerr_kernel<<<blocks, 256, 0, st>>>(Y, s.c, total);
  }
  LDBP_CUDA_TRY(cudaGetLastError());
  return LDBP_OK;
}
