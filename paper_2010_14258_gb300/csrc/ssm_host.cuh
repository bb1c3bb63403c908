// Host-side split-step programs (FP64 tables) and their per-device cache.
#pragma once

#include <complex>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ldbp.h"
#include "ssm.cuh"

namespace ldbp {

struct FiberSI {
  double alpha, beta2, gamma;  // 1/m (power), s^2/m, 1/(W m)
};
FiberSI to_si(const ldbp_fiber& f);
double leff(double alpha, double z);
double lmid(double alpha, double z);

// Spectral tables (DFT order, 1/n folded in) and steps of one split-step run.
struct SsmProgram {
  std::vector<std::vector<std::complex<double>>> tabs;
  std::vector<SsmStep> steps;
  double c_pre = 0.0;
  double noise_std = 0.0;
};

SsmProgram build_channel(const ldbp_fiber& f, const ldbp_link& l, double fs, long long n);
SsmProgram build_dbp(const ldbp_fiber& f, const ldbp_link& l, double fs, long long n, int steps_per_span,
                     bool symmetric);

struct DeviceProgram {
  std::vector<float2*> tabs;        // float heads, [n] each
  std::vector<uint32_t*> tabs_lo;   // tails as half2 bits in units of tabs_lo_scale, [n] each
  std::vector<float> tabs_lo_scale;
  std::vector<SsmStep> host_steps;
  SsmStep* steps = nullptr;
  int nsteps = 0;
  float c_pre = 0.f, noise_std = 0.f;
  // transposed copies of tabs / tabs_lo for the L2-resident path (made on first use)
  std::vector<float2*> st_tabs;
  std::vector<uint32_t*> st_tabs_lo;
};

int get_program(const std::string& key, const SsmProgram& prog, std::shared_ptr<DeviceProgram>* out);
// Cached program of the channel (dbp_steps == 0) or of DBP; tables built on a miss.
int link_program(const ldbp_fiber& f, const ldbp_link& l, double fs, long long n, int dbp_steps, bool dbp_symmetric,
                 std::shared_ptr<DeviceProgram>* out);
// Argument checks of the split-step entry points.  pow2: n must be in the
// fused kernel's range (2^9..2^17, or 3 * 2^9..3 * 2^14); otherwise any n in
// [2, 2^27] (library FFT).
int check_link(const ldbp_fiber* f, const ldbp_link* l, double fs, const void* x, const void* y, long long n,
               int batch, bool pow2 = true);
int get_twiddle(long long n, int P, int log_n2, float2** out);
int run_program(const DeviceProgram& dp, const void* x, void* y, long long n, int batch, const float* wave_scale,
                int wave_mode, uint64_t seed, uint64_t counter, cudaStream_t st);
// L2-resident two-kernel split step (ssm_stream.cu): lengths it supports and the run.
bool ssm_stream_preferred(long long n, int batch);
int run_program_stream(const DeviceProgram& dp, const void* x, void* y, long long n, int batch, uint64_t seed,
                       uint64_t counter, cudaStream_t st);

}  // namespace ldbp
