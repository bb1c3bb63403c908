// Transmitter (Eq. (11)) and receiver chain (Eq. (12)) kernels: RRC pulse
// shaping and matched filtering run as one-step spectral programs of the
// split-step kernel; this file holds the upsampling, the per-waveform
// phase/MSE reduction and the gradient of the MSE loss.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ssm.cuh"
#include "ssm_host.cuh"

namespace ldbp {

// x[b, m] = s[b, m / sps] at m % sps == 0, else 0.
__global__ void upsample_kernel(const float2* __restrict__ s, float2* __restrict__ x, long long nsym, int sps,
                                long long total) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total;
       m += (long long)gridDim.x * blockDim.x) {
    const long long b = m / (nsym * sps), mm = m - b * nsym * sps;
    x[m] = (mm % sps == 0) ? s[b * nsym + mm / sps] : make_float2(0.f, 0.f);
  }
}

// One block per waveform: s_tilde_i = z[b, sps i]; phi = arg(sum conj(s_i) s_tilde_i);
// mse = (sum |s_tilde|^2 + sum |s|^2 - 2 |sum conj(s) s_tilde|) / nsym  (the
// minimum over the common rotation, i.e. ||s_tilde e^{-j phi} - s||^2 / nsym).
template <int NT>
__global__ void __launch_bounds__(NT) rx_stats_kernel(const float2* __restrict__ z, const float2* __restrict__ s,
                                                      long long nsym, int sps, double* __restrict__ stats,
                                                      float* __restrict__ phi) {
  const int b = blockIdx.x;
  const float2* zb = z + (long long)b * nsym * sps;
  const float2* sb = s + (long long)b * nsym;
  double a0 = 0, a1 = 0, dr = 0, di = 0;
  for (long long i = threadIdx.x; i < nsym; i += NT) {
    const float2 zt = zb[i * sps], st = sb[i];
    a0 += (double)zt.x * zt.x + (double)zt.y * zt.y;
    a1 += (double)st.x * st.x + (double)st.y * st.y;
    dr += (double)st.x * zt.x + (double)st.y * zt.y;  // Re conj(s) z
    di += (double)st.x * zt.y - (double)st.y * zt.x;  // Im conj(s) z
  }
  __shared__ double red[4][NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    dr += __shfl_xor_sync(0xffffffffu, dr, o);
    di += __shfl_xor_sync(0xffffffffu, di, o);
  }
  if (lane == 0) {
    red[0][w] = a0;
    red[1][w] = a1;
    red[2][w] = dr;
    red[3][w] = di;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
    for (int i = 0; i < NT / 32; ++i) {
      t0 += red[0][i];
      t1 += red[1][i];
      t2 += red[2][i];
      t3 += red[3][i];
    }
    const double mag = sqrt(t2 * t2 + t3 * t3);
    stats[2 * b] = fmax(t0 + t1 - 2.0 * mag, 0.0) / (double)nsym;
    stats[2 * b + 1] = t1 / (double)nsym;
    phi[b] = (float)atan2(t3, t2);
  }
}

// g[b, sps i] = gscale (s_tilde_i e^{-j phi} - s_i) e^{j phi}, zero elsewhere (in place over z).
__global__ void rx_grad_kernel(float2* __restrict__ z, const float2* __restrict__ s, const float* __restrict__ phi,
                               long long nsym, int sps, float gscale, long long total) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total;
       m += (long long)gridDim.x * blockDim.x) {
    const long long b = m / (nsym * sps), mm = m - b * nsym * sps;
    if (mm % sps != 0) {
      z[m] = make_float2(0.f, 0.f);
      continue;
    }
    const float2 zt = z[m], st = s[b * nsym + mm / sps];
    float sn, cs;
    sincosf(phi[b], &sn, &cs);
    // (z e^{-j phi} - s) e^{j phi} = z - s e^{j phi}
    const float2 se = make_float2(st.x * cs - st.y * sn, st.x * sn + st.y * cs);
    z[m] = make_float2(gscale * (zt.x - se.x), gscale * (zt.y - se.y));
  }
}

// RRC table sqrt(sps RC(f / R_s)) / n on the fftfreq grid.
static std::vector<std::complex<double>> rrc_table(long long n, int sps, double beta) {
  std::vector<std::complex<double>> t((size_t)n);
  const double lo = (1.0 - beta) / 2.0, hi = (1.0 + beta) / 2.0, pi = 3.14159265358979323846;
  for (long long k = 0; k < n; ++k) {
    const double kk = (double)(k < (n + 1) / 2 ? k : k - n);
    const double a = std::fabs(kk / (double)n * sps);
    double rc = 0.0;
    if (a <= lo) rc = 1.0;
    else if (a <= hi) rc = 0.5 * (1.0 + std::cos(pi / beta * (a - lo)));
    t[(size_t)k] = std::sqrt(sps * rc) / (double)n;
  }
  return t;
}

static int rrc_program(long long n, int sps, double beta, double step_scale, std::shared_ptr<DeviceProgram>* dp) {
  char key[128];
  snprintf(key, sizeof(key), "rrc|%lld,%d,%.17g,%.17g", n, sps, beta, step_scale);
  SsmProgram prog;
  prog.tabs.push_back(rrc_table(n, sps, beta));
  prog.steps.push_back({0, -2, 0, (float)step_scale, 0.0f});
  return get_program(key, prog, dp);
}

static int check_txrx(long long nsym, int sps, double beta, int batch) {
  if (sps < 1 || nsym < 1 || batch < 1) return fail(LDBP_EINVAL, "nsym, sps and batch must be >= 1");
  if (!(beta > 0.0 && beta <= 1.0)) return fail(LDBP_EINVAL, "rolloff must be in (0, 1]");
  const long long n = nsym * sps;
  if (n & (n - 1)) return fail(LDBP_EINVAL, "n = nsym * sps = %lld must be a power of two", n);
  return 0;
}

}  // namespace ldbp

using namespace ldbp;

extern "C" {

int ldbp_tx(const void* symbols, const float* power_w, int32_t sps, double rolloff, void* x, int64_t nsym,
            int32_t batch, void* stream) {
  if (!symbols || !power_w || !x) return fail(LDBP_EINVAL, "symbols, power_w and x must be non-NULL");
  if (int rc = check_txrx(nsym, sps, rolloff, batch)) return rc;
  const long long n = nsym * sps, total = n * batch;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::shared_ptr<DeviceProgram> dp;
  if (int rc = rrc_program(n, sps, rolloff, std::sqrt((double)sps), &dp)) return rc;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 65536);
  upsample_kernel<<<blocks, 256, 0, st>>>(static_cast<const float2*>(symbols), static_cast<float2*>(x), nsym, sps,
                                          total);
  LDBP_CUDA_TRY(cudaGetLastError());
  return run_program(*dp, x, x, n, batch, power_w, 1, 0, 0, st);
}

int ldbp_rx(const void* y, const void* symbols, const float* power_w, int32_t sps, double rolloff, int64_t nsym,
            int32_t batch, double* stats, float* phi, void* grad, float grad_scale, void* workspace, void* stream) {
  if (!y || !symbols || !power_w || !stats || !phi || !workspace)
    return fail(LDBP_EINVAL, "y, symbols, power_w, stats, phi and workspace must be non-NULL");
  if (int rc = check_txrx(nsym, sps, rolloff, batch)) return rc;
  const long long n = nsym * sps, total = n * batch;
  if (grad && (grad == y || grad == workspace)) return fail(LDBP_EINVAL, "grad must not alias y or workspace");
  if (workspace == y) return fail(LDBP_EINVAL, "workspace must not alias y");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::shared_ptr<DeviceProgram> dp;
  if (int rc = rrc_program(n, sps, rolloff, 1.0 / std::sqrt((double)sps), &dp)) return rc;
  if (int rc = run_program(*dp, y, workspace, n, batch, power_w, 2, 0, 0, st)) return rc;
  rx_stats_kernel<256><<<batch, 256, 0, st>>>(static_cast<const float2*>(workspace),
                                              static_cast<const float2*>(symbols), nsym, sps, stats, phi);
  LDBP_CUDA_TRY(cudaGetLastError());
  if (grad) {
    const int blocks = (int)std::min<long long>((total + 255) / 256, 65536);
    rx_grad_kernel<<<blocks, 256, 0, st>>>(static_cast<float2*>(workspace), static_cast<const float2*>(symbols),
                                           phi, nsym, sps, grad_scale, total);
    LDBP_CUDA_TRY(cudaGetLastError());
    if (int rc = run_program(*dp, workspace, grad, n, batch, power_w, 2, 0, 0, st)) return rc;
  }
  return LDBP_OK;
}

}  // extern "C"
