// Receiver front end of Sec. IV-A: the channel is simulated at rho_a
// samples/symbol, then the received waveform passes an ideal brick-wall
// low-pass of total bandwidth Delta B and is sampled at the DSP rate f_s.  The
// same band limit run the other way is band-limited interpolation of a
// DSP-rate waveform (e.g. a transmit waveform) onto the analog grid.
//
// Both grids span one period N_sym / R_s, so DFT bin kappa is the same
// frequency on either and the whole operation is: a forward FFT on the input
// grid, a gather of the passband bins |kappa| <= kmax into the output grid's
// DFT order (scaled by 1 / n_in, every other output bin zero), and an inverse
// FFT on the output grid.  The transforms are cuFFT (any length, e.g. the
// 6 samples/symbol grids); the gather is the kernel below.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "cufft_plan.cuh"

namespace ldbp {

// Y[b][j] = X[b][kappa mod n_in] * scale when |kappa| <= kmax, else 0, where
// kappa is output bin j in signed (fftfreq) order.  kmax < n_in / 2 and
// kmax < n_out / 2, so each kept bin has a unique source in [0, n_in).
__global__ void band_gather_kernel(const float2* __restrict__ X, float2* __restrict__ Y, long long n_in,
                                   long long n_out, long long kmax, float scale, long long total) {
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < total;
       m += (long long)gridDim.x * blockDim.x) {
    const long long b = m / n_out, j = m - b * n_out;
    const long long kappa = j < (n_out + 1) / 2 ? j : j - n_out;
    float2 v = make_float2(0.f, 0.f);
    if (kappa <= kmax && -kappa <= kmax) {
      const float2 x = X[b * n_in + (kappa >= 0 ? kappa : kappa + n_in)];
      v = make_float2(x.x * scale, x.y * scale);
    }
    Y[m] = v;
  }
}

static bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + bbytes && pb < pa + abytes;
}

// Largest integer kappa with kappa < bandwidth * n_coarse / 2 (the open
// passband), evaluated in double in that order.
static long long passband_kmax(double bandwidth, long long n_coarse) {
  const double edge = bandwidth * (double)n_coarse / 2.0;
  return (long long)std::ceil(edge) - 1;
}

}  // namespace ldbp

using namespace ldbp;

extern "C" {

size_t ldbp_resample_workspace(int64_t n_in, int32_t batch) {
  if (n_in < 2 || batch < 1) return 0;
  return (size_t)n_in * (size_t)batch * sizeof(float2);
}

int ldbp_resample(const void* x, int64_t n_in, void* y, int64_t n_out, double bandwidth, int32_t batch,
                  void* workspace, size_t workspace_bytes, void* stream) {
  if (!x || !y || !workspace) return fail(LDBP_EINVAL, "x, y and workspace must be non-NULL");
  if (!std::isfinite(bandwidth)) return fail(LDBP_ENONFINITE, "bandwidth is NaN or infinite");
  if (!(bandwidth > 0.0 && bandwidth <= 1.0)) return fail(LDBP_EINVAL, "bandwidth must be in (0, 1]");
  if (n_in < 2 || n_out < 2 || n_in > (1LL << 27) || n_out > (1LL << 27))
    return fail(LDBP_EINVAL, "n_in=%lld and n_out=%lld must be in [2, 2^27]", (long long)n_in, (long long)n_out);
  if (n_in % n_out != 0 && n_out % n_in != 0)
    return fail(LDBP_EINVAL, "one of n_in=%lld, n_out=%lld must divide the other", (long long)n_in,
                (long long)n_out);
  if (batch < 1) return fail(LDBP_EINVAL, "batch=%d must be >= 1", batch);
  const size_t in_bytes = (size_t)n_in * (size_t)batch * sizeof(float2);
  const size_t out_bytes = (size_t)n_out * (size_t)batch * sizeof(float2);
  if (workspace_bytes < in_bytes)
    return fail(LDBP_EINVAL, "workspace of %zu bytes, need %zu", workspace_bytes, in_bytes);
  if (!aligned16(workspace) || !aligned16(x) || !aligned16(y))
    return fail(LDBP_EINVAL, "x, y and workspace must be 16-byte aligned");
  if (overlaps(workspace, in_bytes, x, in_bytes) || overlaps(workspace, in_bytes, y, out_bytes))
    return fail(LDBP_EINVAL, "workspace overlaps x or y");
  const long long kmax = passband_kmax(bandwidth, n_in < n_out ? n_in : n_out);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cufftHandle fwd, inv;
  if (int rc = cufft_plan(n_in, batch, st, &fwd)) return rc;
  if (int rc = cufft_plan(n_out, batch, st, &inv)) return rc;
  float2* W = static_cast<float2*>(workspace);
  float2* Y = static_cast<float2*>(y);
  if (cufftExecC2C(fwd, (cufftComplex*)const_cast<void*>(x), (cufftComplex*)W, CUFFT_FORWARD) != CUFFT_SUCCESS)
    return fail(LDBP_ECUDA, "cufftExecC2C forward failed");
  const long long total = n_out * (long long)batch;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
  band_gather_kernel<<<blocks, 256, 0, st>>>(W, Y, n_in, n_out, kmax, (float)(1.0 / (double)n_in), total);
  LDBP_CUDA_TRY(cudaGetLastError());
  if (cufftExecC2C(inv, (cufftComplex*)Y, (cufftComplex*)Y, CUFFT_INVERSE) != CUFFT_SUCCESS)
    return fail(LDBP_ECUDA, "cufftExecC2C inverse failed");
  return LDBP_OK;
}

}  // extern "C"
