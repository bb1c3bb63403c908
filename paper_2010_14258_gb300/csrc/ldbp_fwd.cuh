// Internal interface of the fused learned-DBP kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ldbp.h"

namespace ldbp {

// Default register-tile geometry (the adjoint, the filtered-power kernels and
// the forward instances with K <= 2 or K <= 16 dispatch); the other forward
// and ragged instances use 32 samples per thread in 128-thread blocks.
constexpr int kFwdR = 16;                 // consecutive samples held by one thread
constexpr int kFwdNT = 256;               // threads per block
constexpr int kFwdNW = kFwdNT / 32;       // warps per block
constexpr int kFwdS = kFwdR * kFwdNT;     // samples per tile (incl. halo)
constexpr int kFwdEdge = LDBP_MAX_HALF_TAPS;

struct FwdParams {
  const float2* x;
  float2* y;
  float2* ckpt;          // [M][batch][n] or nullptr
  const float2* taps;    // [M][taps_stride]
  int taps_stride;
  long long n;
  int batch;
  int M;
  int tiles_per_wave;
  int L;                 // output samples per tile (even)
  int Hp;                // halo per side (even, >= sum K_i)
  int K[LDBP_MAX_STEPS];
  float c[LDBP_MAX_STEPS];
};

// Tile plan shared by the forward and adjoint kernels.
struct TilePlan {
  int Hp, L, tiles_per_wave;
};
int make_tile_plan(long long n, int H, TilePlan* out, int S = kFwdS);

cudaError_t launch_ldbp_fwd(const FwdParams& p, int kmax_needed, cudaStream_t st);
size_t fwd_smem_bytes(int kmax, int M, int S);
// Tile size (samples) of the forward instance chosen for these step widths.
int fwd_tile_samples(const int* K, int M, int kmax_needed);
int fwd_kmax_class(int kmax_needed);

}  // namespace ldbp
