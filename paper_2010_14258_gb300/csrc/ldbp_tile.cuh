// Register-tile helpers shared by the fused learned-DBP kernels: each thread
// holds kFwdR consecutive samples; neighbours come from adjacent lanes by warp
// shuffles and from adjacent warps through a small shared-memory edge buffer.
#pragma once

#include "common.cuh"
#include "ldbp_fwd.cuh"

namespace ldbp {

// xe[0..K) = the K samples left of v, xe[K..K+R) = v, xe[K+R..K+R+K) = the K
// samples right of v.  The first (last) warp of the block sees zeros beyond
// the tile.  Contains one __syncthreads (edge exchange between warps).
template <int K>
__device__ __forceinline__ void tile_extend(const float2 (&v)[kFwdR], float2 (&xe)[kFwdR + 2 * K], float2* edge_first,
                                            float2* edge_last, int lane, int warp) {
  if constexpr (K > 0) {
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < K; ++j) edge_first[warp * kFwdEdge + j] = v[j];
    }
    if (lane == 31) {
#pragma unroll
      for (int j = 0; j < K; ++j) edge_last[warp * kFwdEdge + j] = v[kFwdR - K + j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      xe[j].x = __shfl_up_sync(0xffffffffu, v[kFwdR - K + j].x, 1);
      xe[j].y = __shfl_up_sync(0xffffffffu, v[kFwdR - K + j].y, 1);
      xe[K + kFwdR + j].x = __shfl_down_sync(0xffffffffu, v[j].x, 1);
      xe[K + kFwdR + j].y = __shfl_down_sync(0xffffffffu, v[j].y, 1);
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        xe[j] = warp > 0 ? edge_last[(warp - 1) * kFwdEdge + j] : make_float2(0.f, 0.f);
    }
    if (lane == 31) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        xe[K + kFwdR + j] = warp < kFwdNW - 1 ? edge_first[(warp + 1) * kFwdEdge + j] : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int r = 0; r < kFwdR; ++r) xe[K + r] = v[r];
}

// out[r] = h_0 xe[K+r] + sum_k h_k (xe[K+r-k] + xe[K+r+k])   (folded symmetric FIR);
// with CONJ the taps are conjugated (the adjoint filter).
template <int K, bool CONJ>
__device__ __forceinline__ void tile_fir(const float2 (&xe)[kFwdR + 2 * K], const float2* __restrict__ h,
                                         float2 (&out)[kFwdR]) {
  float2 hk[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    hk[k] = h[k];
    if (CONJ) hk[k].y = -hk[k].y;
  }
#pragma unroll
  for (int r = 0; r < kFwdR; ++r) {
    const float2 x0 = xe[K + r];
    float2 acc = make_float2(fmaf(hk[0].x, x0.x, -hk[0].y * x0.y), fmaf(hk[0].x, x0.y, hk[0].y * x0.x));
#pragma unroll
    for (int k = 1; k <= K; ++k) acc = cfma(hk[k], cadd(xe[K + r - k], xe[K + r + k]), acc);
    out[r] = acc;
  }
}

// e[r] = exp(j c |v[r]|^2).  A warp whose phases all lie in [-pi/4, pi/4]
// skips the range reduction; the results are identical either way.
__device__ __forceinline__ void tile_expj(const float2 (&v)[kFwdR], float c, float2 (&e)[kFwdR]) {
  float phi[kFwdR];
  float m = 0.f;
#pragma unroll
  for (int r = 0; r < kFwdR; ++r) {
    phi[r] = c * fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
    m = fmaxf(m, fabsf(phi[r]));
  }
  if (__all_sync(0xffffffffu, m <= 0.785398163f)) {
#pragma unroll
    for (int r = 0; r < kFwdR; ++r) e[r] = expj<false>(phi[r]);
  } else {
#pragma unroll
    for (int r = 0; r < kFwdR; ++r) e[r] = expj<true>(phi[r]);
  }
}

}  // namespace ldbp
