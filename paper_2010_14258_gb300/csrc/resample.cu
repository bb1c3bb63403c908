// Receiver front end of Sec. IV-A: the channel is simulated at rho_a
// samples/symbol, then the received waveform passes an ideal brick-wall
// low-pass of total bandwidth Delta B and is sampled at the DSP rate f_s.  The
// same band limit run the other way is band-limited interpolation of a
// DSP-rate waveform (e.g. a transmit waveform) onto the analog grid.
//
// Both grids span one period N_sym / R_s, so DFT bin kappa is the same
// frequency on either.  With the fine grid n_f = r n_c (n_c the coarse grid)
// and its polyphase rows x_p[q] = x[r q + p] (p < r, q < n_c):
//   X[kappa] = sum_p e^{-j 2 pi kappa p / n_f} DFT_{n_c}(x_p)[kappa mod n_c],
// so sampling down is r transforms of length n_c, a twiddled sum over p on
// the passband bins |kappa| <= kmax (scaled by 1 / n_in, every other bin zero) and one
// inverse transform of length n_c; interpolation is the same run backwards
// (one transform, r twiddled inverse transforms, output row p to samples
// r q + p).  One block per waveform does all of it in shared memory with the
// split-step kernel's Stockham passes, so the input is read once and the
// output written once: 8 (n_f + n_c) bytes per waveform, the algorithmic
// traffic of the operation.
#include <algorithm>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "ssm_host.cuh"
#include "ssm_kernel.cuh"

namespace ldbp {

constexpr int kRsMinLog = 9, kRsMaxLog = 12, kRsMaxRatio = 8;
constexpr long long kRsMaxFine = 16384;  // r n_c: the r rows must fit in shared memory

// e^{-j 2 pi kappa_k p / n_f} for p = 1..r-1 and every coarse bin k (signed
// kappa_k, fftfreq order), [(p - 1) n_c + k]; cached per (device, n_c, r).
static std::mutex g_rs_mu;
static std::map<std::string, float2*> g_rs_phase;

static int rs_phase(int n_c, int r, float2** out) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  const std::string key = std::to_string(dev) + ":" + std::to_string(n_c) + ":" + std::to_string(r);
  std::lock_guard<std::mutex> lk(g_rs_mu);
  auto it = g_rs_phase.find(key);
  if (it != g_rs_phase.end()) {
    *out = it->second;
    return 0;
  }
  const double pi = 3.14159265358979323846;
  std::vector<float2> h((size_t)std::max(1, r - 1) * (size_t)n_c, make_float2(1.f, 0.f));
  for (int p = 1; p < r; ++p)
    for (int k = 0; k < n_c; ++k) {
      const long long kap = k < n_c / 2 ? k : k - n_c;
      const double a = -2.0 * pi * (double)(kap * p) / ((double)n_c * r);
      h[(size_t)(p - 1) * n_c + k] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
  float2* d = nullptr;
  cudaError_t e = cudaMalloc(&d, h.size() * sizeof(float2));
  if (e != cudaSuccess) return cuda_fail(e, "resample phase table");
  e = cudaMemcpy(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "resample phase table copy");
  g_rs_phase[key] = d;
  *out = d;
  return 0;
}

struct RsParams {
  const float2* x;
  float2* y;
  const float2* twiddle;  // local-transform twiddles of n_c (get_twiddle with P = 1), read through L1
  const float2* phase;    // rs_phase table
  int r;                  // n_f / n_c
  int groups;             // thread groups of n_c / 16 threads; each transforms rows g, g + groups, ...
  int kmax;               // passband |kappa| <= kmax
  float scale;            // 1 / n_in
};

constexpr int kRsMaxThreads = 512;

// DOWN: x [batch][r n_c] -> y [batch][n_c];  !DOWN: x [batch][n_c] -> y [batch][r n_c].
// The block has `groups` thread groups of N / 16 threads; the r polyphase
// transforms run one row per group at a time (concurrently when groups > 1).
template <int LOGN, bool DOWN>
__global__ void __launch_bounds__(kRsMaxThreads) resample_kernel(const __grid_constant__ RsParams p) {
  constexpr int N = 1 << LOGN, NT = N / kSsmE, ROW = N + N / 16;
  extern __shared__ __align__(16) float2 rows[];  // r rows of [spad(N)]
  const int tid = threadIdx.x, nthr = blockDim.x, g = tid / NT, t = tid - g * NT;
  const int b = blockIdx.x, r = p.r, G = p.groups, rounds = (r + G - 1) / G;
  const int nf = r * N;
  const float2* __restrict__ tw = p.twiddle;
  if constexpr (DOWN) {
    // polyphase rows of the fine-grid waveform (coalesced reads)
    const float2* __restrict__ xin = p.x + (long long)b * nf;
    for (int m = tid; m < nf; m += nthr) {
      const int q = m / r, ph = m - q * r;
      rows[ph * ROW + spad(q)] = xin[m];
    }
    __syncthreads();
    for (int k = 0; k < rounds; ++k) {
      const int ph = g + k * G;
      ssm_local_fft<LOGN, 0>(rows + (ph < r ? ph : 0) * ROW, tw, t, ph < r);
    }
    // passband bins: Z[k] = scale sum_p phase_p[k] Y_p[k]; conjugated for the inverse
    for (int k = tid; k < N; k += nthr) {
      const int kap = k < N / 2 ? k : k - N;
      float2 z = make_float2(0.f, 0.f);
      if (kap <= p.kmax && -kap <= p.kmax) {
        z = rows[spad(k)];
        for (int ph = 1; ph < r; ++ph) z = cadd(z, cmul(rows[ph * ROW + spad(k)], __ldg(&p.phase[(ph - 1) * N + k])));
        z = make_float2(z.x * p.scale, -z.y * p.scale);
      }
      rows[spad(k)] = z;
    }
    __syncthreads();
    ssm_local_ifft<LOGN, ssm_npass(LOGN) - 1>(rows, tw, 0.f, t, g == 0);
    float2* __restrict__ yout = p.y + (long long)b * N;
    for (int m = tid; m < N; m += nthr) yout[m] = rows[spad(m)];
  } else {
    const float2* __restrict__ xin = p.x + (long long)b * N;
    for (int m = tid; m < N; m += nthr) rows[spad(m)] = xin[m];
    __syncthreads();
    ssm_local_fft<LOGN, 0>(rows, tw, t, g == 0);
    // row p holds conj(scale e^{+j 2 pi kappa p / n_f} X[k]) on the passband (scale = 1 / n_c)
    for (int k = tid; k < N; k += nthr) {
      const int kap = k < N / 2 ? k : k - N;
      const bool pass = kap <= p.kmax && -kap <= p.kmax;
      const float2 v = rows[spad(k)];
      const float2 z = pass ? make_float2(v.x * p.scale, v.y * p.scale) : make_float2(0.f, 0.f);
      for (int ph = 1; ph < r; ++ph) {
        const float2 w = cmulc(z, __ldg(&p.phase[(ph - 1) * N + k]));
        rows[ph * ROW + spad(k)] = make_float2(w.x, -w.y);
      }
      rows[spad(k)] = make_float2(z.x, -z.y);
    }
    __syncthreads();
    for (int k = 0; k < rounds; ++k) {
      const int ph = g + k * G;
      ssm_local_ifft<LOGN, ssm_npass(LOGN) - 1>(rows + (ph < r ? ph : 0) * ROW, tw, 0.f, t, ph < r);
    }
    float2* __restrict__ yout = p.y + (long long)b * nf;
    for (int m = tid; m < nf; m += nthr) {
      const int q = m / r, ph = m - q * r;
      yout[m] = rows[ph * ROW + spad(q)];
    }
  }
}

template <int LOGN, bool DOWN>
static cudaError_t rs_launch(RsParams p, int batch, cudaStream_t st) {
  constexpr int N = 1 << LOGN, NT = N / kSsmE;
  // thread groups only to give short grids at least 128 threads per block: the
  // passes need 128 registers a thread, so blocks of N / 16 threads (4 per SM
  // at N = 2048) keep more independent work on an SM than one wide block
  p.groups = std::max(1, std::min(p.r, 128 / NT));
  const size_t smem = sizeof(float2) * (size_t)p.r * (N + N / 16);
  auto kern = resample_kernel<LOGN, DOWN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<batch, p.groups * NT, smem, st>>>(p);
  return cudaGetLastError();
}

static cudaError_t rs_dispatch(const RsParams& p, int log_c, bool down, int batch, cudaStream_t st) {
  switch (log_c) {
    case 9: return down ? rs_launch<9, true>(p, batch, st) : rs_launch<9, false>(p, batch, st);
    case 10: return down ? rs_launch<10, true>(p, batch, st) : rs_launch<10, false>(p, batch, st);
    case 11: return down ? rs_launch<11, true>(p, batch, st) : rs_launch<11, false>(p, batch, st);
    case 12: return down ? rs_launch<12, true>(p, batch, st) : rs_launch<12, false>(p, batch, st);
    default: return cudaErrorInvalidValue;
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

int ldbp_resample(const void* x, int64_t n_in, void* y, int64_t n_out, double bandwidth, int32_t batch,
                  void* stream) {
  if (!x || !y) return fail(LDBP_EINVAL, "x and y must be non-NULL");
  if (!std::isfinite(bandwidth)) return fail(LDBP_ENONFINITE, "bandwidth is NaN or infinite");
  if (!(bandwidth > 0.0 && bandwidth <= 1.0)) return fail(LDBP_EINVAL, "bandwidth must be in (0, 1]");
  if (batch < 1) return fail(LDBP_EINVAL, "batch=%d must be >= 1", batch);
  if (n_in < 1 || n_out < 1 || (n_in % n_out != 0 && n_out % n_in != 0))
    return fail(LDBP_EINVAL, "one of n_in=%lld, n_out=%lld must divide the other", (long long)n_in,
                (long long)n_out);
  const bool down = n_in >= n_out;
  const long long nc = down ? n_out : n_in, nf = down ? n_in : n_out, r = nf / nc;
  int log_c = 0;
  while ((1LL << log_c) < nc) ++log_c;
  if ((1LL << log_c) != nc || log_c < kRsMinLog || log_c > kRsMaxLog || r > kRsMaxRatio || nf > kRsMaxFine)
    return fail(LDBP_EINVAL,
                "coarse grid %lld must be a power of two in [%d, %d], the ratio at most %d and the fine grid at "
                "most %lld samples",
                nc, 1 << kRsMinLog, 1 << kRsMaxLog, kRsMaxRatio, kRsMaxFine);
  if (!aligned16(x) || !aligned16(y)) return fail(LDBP_EINVAL, "x and y must be 16-byte aligned");
  const size_t in_bytes = (size_t)n_in * (size_t)batch * sizeof(float2);
  const size_t out_bytes = (size_t)n_out * (size_t)batch * sizeof(float2);
  if (!(x == y && n_in == n_out) && overlaps(x, in_bytes, y, out_bytes))
    return fail(LDBP_EINVAL, "x and y overlap (only y == x with n_in == n_out is allowed)");
  RsParams p;
  p.x = static_cast<const float2*>(x);
  p.y = static_cast<float2*>(y);
  p.r = (int)r;
  p.kmax = (int)passband_kmax(bandwidth, nc);
  p.scale = (float)(1.0 / (double)n_in);
  float2* tw = nullptr;
  if (int rc = get_twiddle(nc, 1, log_c, &tw)) return rc;
  float2* ph = nullptr;
  if (int rc = rs_phase((int)nc, (int)r, &ph)) return rc;
  p.twiddle = tw;
  p.phase = ph;
  cudaError_t e = rs_dispatch(p, log_c, down, batch, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "resample launch");
  return LDBP_OK;
}

}  // extern "C"
