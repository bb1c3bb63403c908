// Internal interface of the cluster-resident split-step Fourier kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ldbp {

// One split-step "program step": spectral multiply (and optional ASE add),
// inverse transform, Kerr rotation.  In the spectral domain
//   X' = scale * tab[k] * X + [noise] noise_tab[k] * noise_std * g_k(span)
// where each table value is a float head (tabs) plus a tail (tabs_lo: the
// remainder as a half2, in units of tabs_lo_scale)
// (noise_tab == -1 means a flat 1/n), then u = iDFT(X') (1/n folded into the
// tables) and u <- u exp(j c |u|^2) when c != 0.
struct SsmStep {
  int16_t tab;
  int16_t noise_tab;   // -2: no noise, -1: flat 1/n, >= 0: table index
  int32_t span;        // ASE counter word
  float scale;
  float c;
};

constexpr int kSsmMaxTabs = 4;

struct SsmParams {
  const float2* x;
  float2* y;
  long long n;
  int batch;
  int nsteps;
  const SsmStep* steps;                 // device [nsteps]
  const float2* tabs[kSsmMaxTabs];      // device [n] each, DFT order: float head of each value
  const uint32_t* tabs_lo[kSsmMaxTabs]; // device [n] each: tail (value - head) / tabs_lo_scale as half2 bits
  float tabs_lo_scale[kSsmMaxTabs];
  const float2* twiddle;                // device twiddle buffer (layout in ssm_kernel.cuh)
  const float* wave_scale;              // device [batch] per-waveform factor of step 0, or nullptr
  int wave_mode;                        // factor = w, sqrt(w) or 1/sqrt(w) for mode 0, 1, 2
  float c_pre;                          // Kerr applied to the input before step 0 (0: none)
  float noise_std;                      // sqrt(n sigma^2 / 2)
  uint32_t seed_lo, seed_hi, counter;
};

// Number of twiddle entries for (P, N2).
long long ssm_twiddle_count(int P, int log_n2);
// Launches the kernel for waveform length n = P * N2 (both powers of two).
cudaError_t launch_ssm(const SsmParams& p, int P, int log_n2, cudaStream_t st);
// Largest supported per-block length and cluster size.
constexpr int kSsmMaxLogN2 = 13;
constexpr int kSsmMaxCluster = 16;
constexpr int kSsmMinLogN2 = 9;
// Chooses the cluster size for a batch of waveforms of length n (power of two).
int ssm_choose_cluster(long long n, int batch, int sm_count, int* P, int* log_n2);

}  // namespace ldbp
