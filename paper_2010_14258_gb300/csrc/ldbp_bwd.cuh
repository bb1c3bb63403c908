// Internal interface of the learned-DBP adjoint kernels.
#pragma once

#include <cuda_runtime.h>

#include "ldbp_fwd.cuh"

namespace ldbp {

struct BwdParams {
  const float2* ckpt;    // [M][batch][n]: input of every step
  const float2* gy;      // [batch][n]
  float2* gx;            // [batch][n] or nullptr
  float2* partial;       // [blocks][M][KMAX+2] per-block tap sums, then the c-gradient sum
  const float2* taps;
  int taps_stride;
  long long n;
  int batch;
  int M;
  int tiles_per_wave;
  int L;
  int Hp;
  int K[LDBP_MAX_STEPS];
  float c[LDBP_MAX_STEPS];
};

struct TapReduceK {
  int K[LDBP_MAX_STEPS];
};

cudaError_t launch_ldbp_bwd(const BwdParams& p, int kmax_class, cudaStream_t st);
// ldbp_bwd_fix_kernel (ldbp_bwd_fix.cu) runs every model except the mixed
// ones with a filter wider than T = 17: bwd_fixed_width returns the instance
// to launch (class * kFixSel + K for one width K in every step, class *
// kFixSel + kFixMixed for mixed widths), else -1 (ldbp_bwd_kernel).
constexpr int kFixSel = 32, kFixMixed = 31;
int bwd_fixed_width(const BwdParams& p);
cudaError_t launch_ldbp_bwd_fixed(const BwdParams& p, int sel, cudaStream_t st);
cudaError_t launch_tap_reduce(const float2* partial, int tiles, int M, int pstride, const TapReduceK& kk,
                              float2* gtaps, int taps_stride, cudaStream_t st);
cudaError_t launch_c_reduce(const float2* partial, int tiles, int M, int pstride, float* gc, cudaStream_t st);
size_t bwd_smem_bytes(int kmax, int M);

}  // namespace ldbp
