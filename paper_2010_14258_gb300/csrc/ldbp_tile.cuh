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

// Taps pre-expanded for packed FP32x2 arithmetic: (h.re, h.re, h.im, h.im).
__device__ __forceinline__ float4 tap_pair(float2 h) { return make_float4(h.x, h.x, h.y, h.y); }

// out[r] = h_0 xe[K+r] + sum_k h_k (xe[K+r-k] + xe[K+r+k])   (folded symmetric FIR);
// with CONJ the taps are conjugated (the adjoint filter).  Packed FP32x2
// form: A accumulates h.re * (s.re, s.im) and Bv accumulates h.im * (s.re, s.im),
// so h s = (A.re - Bv.im, A.im + Bv.re): 3 packed instructions per tap pair.
template <int K, bool CONJ>
__device__ __forceinline__ void tile_fir(const float2 (&xe)[kFwdR + 2 * K], const float4* __restrict__ h4,
                                         float2 (&out)[kFwdR]) {
  float2 hr[K + 1], hi[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    const float4 q = h4[k];
    hr[k] = make_float2(q.x, q.y);
    hi[k] = make_float2(q.z, q.w);
  }
#pragma unroll
  for (int r = 0; r < kFwdR; ++r) {
    float2 A = __fmul2_rn(hr[0], xe[K + r]);
    float2 Bv = __fmul2_rn(hi[0], xe[K + r]);
#pragma unroll
    for (int k = 1; k <= K; ++k) {
      const float2 sk = __fadd2_rn(xe[K + r - k], xe[K + r + k]);
      A = __ffma2_rn(hr[k], sk, A);
      Bv = __ffma2_rn(hi[k], sk, Bv);
    }
    out[r] = CONJ ? make_float2(A.x + Bv.y, A.y - Bv.x) : make_float2(A.x - Bv.y, A.y + Bv.x);
  }
}

// exp(j phi) for two phases at once (packed FP32x2), |phi| <= pi/4: the
// Taylor polynomials of expj<false> evaluated on (phi_a, phi_b).
__device__ __forceinline__ void expj_pair(float2 phi, float2& c, float2& s) {
  const float2 r2 = __fmul2_rn(phi, phi);
  float2 ps = __ffma2_rn(r2, make_float2(2.75573192239858907e-6f, 2.75573192239858907e-6f),
                         make_float2(-1.98412698412698413e-4f, -1.98412698412698413e-4f));
  ps = __ffma2_rn(r2, ps, make_float2(8.33333333333333333e-3f, 8.33333333333333333e-3f));
  ps = __ffma2_rn(r2, ps, make_float2(-1.66666666666666667e-1f, -1.66666666666666667e-1f));
  s = __ffma2_rn(__fmul2_rn(r2, phi), ps, phi);
  float2 pc = __ffma2_rn(r2, make_float2(-2.75573192239858907e-7f, -2.75573192239858907e-7f),
                         make_float2(2.48015873015873016e-5f, 2.48015873015873016e-5f));
  pc = __ffma2_rn(r2, pc, make_float2(-1.38888888888888889e-3f, -1.38888888888888889e-3f));
  pc = __ffma2_rn(r2, pc, make_float2(4.16666666666666667e-2f, 4.16666666666666667e-2f));
  pc = __ffma2_rn(r2, pc, make_float2(-0.5f, -0.5f));
  c = __ffma2_rn(r2, pc, make_float2(1.0f, 1.0f));
}

// The same for |phi| <= 1/4, where the Taylor series truncated after phi^5
// (sine) and phi^6 (cosine) is below 1.2e-8 and 3.8e-10, under half an FP32
// ulp of the unit-modulus result.
__device__ __forceinline__ void expj_pair_small(float2 phi, float2& c, float2& s) {
  const float2 r2 = __fmul2_rn(phi, phi);
  const float2 ps = __ffma2_rn(r2, make_float2(8.33333333333333333e-3f, 8.33333333333333333e-3f),
                               make_float2(-1.66666666666666667e-1f, -1.66666666666666667e-1f));
  s = __ffma2_rn(__fmul2_rn(r2, phi), ps, phi);
  float2 pc = __ffma2_rn(r2, make_float2(-1.38888888888888889e-3f, -1.38888888888888889e-3f),
                         make_float2(4.16666666666666667e-2f, 4.16666666666666667e-2f));
  pc = __ffma2_rn(r2, pc, make_float2(-0.5f, -0.5f));
  c = __ffma2_rn(r2, pc, make_float2(1.0f, 1.0f));
}

// Phases phi[r] = c |v[r]|^2 of the thread's samples and their maximum magnitude.
__device__ __forceinline__ float tile_phases(const float2 (&v)[kFwdR], float c, float (&phi)[kFwdR]) {
  float m = 0.f;
#pragma unroll
  for (int r = 0; r < kFwdR; r += 2) {
    const float2 a = __fmul2_rn(v[r], v[r]), b = __fmul2_rn(v[r + 1], v[r + 1]);
    const float2 p = __fmul2_rn(make_float2(a.x + a.y, b.x + b.y), make_float2(c, c));
    phi[r] = p.x;
    phi[r + 1] = p.y;
    m = fmaxf(m, fmaxf(fabsf(p.x), fabsf(p.y)));
  }
  return m;
}

// e[r] = exp(j c |v[r]|^2).  The polynomial is chosen per warp from the
// largest phase: |phi| <= 1/4 (the usual case: the nonlinear phase per step
// is small) and |phi| <= pi/4 use packed FP32x2 Taylor polynomials without
// range reduction; larger phases take the reducing scalar path.  Every path
// is accurate to about one FP32 ulp.
__device__ __forceinline__ void tile_expj(const float2 (&v)[kFwdR], float c, float2 (&e)[kFwdR]) {
  float phi[kFwdR];
  const float m = tile_phases(v, c, phi);
  if (__all_sync(0xffffffffu, m <= 0.25f)) {
#pragma unroll
    for (int r = 0; r < kFwdR; r += 2) {
      float2 cc, ss;
      expj_pair_small(make_float2(phi[r], phi[r + 1]), cc, ss);
      e[r] = make_float2(cc.x, ss.x);
      e[r + 1] = make_float2(cc.y, ss.y);
    }
  } else if (__all_sync(0xffffffffu, m <= 0.785398163f)) {
#pragma unroll
    for (int r = 0; r < kFwdR; r += 2) {
      float2 cc, ss;
      expj_pair(make_float2(phi[r], phi[r + 1]), cc, ss);
      e[r] = make_float2(cc.x, ss.x);
      e[r + 1] = make_float2(cc.y, ss.y);
    }
  } else {
#pragma unroll
    for (int r = 0; r < kFwdR; ++r) e[r] = expj<true>(phi[r]);
  }
}

// v[r] <- v[r] exp(j c |v[r]|^2) in place (the Kerr step), without
// materialising the rotation pairs.
__device__ __forceinline__ void tile_kerr(float2 (&v)[kFwdR], float c) {
  float phi[kFwdR];
  const float m = tile_phases(v, c, phi);
  if (__all_sync(0xffffffffu, m <= 0.25f)) {
#pragma unroll
    for (int r = 0; r < kFwdR; r += 2) {
      float2 cc, ss;
      expj_pair_small(make_float2(phi[r], phi[r + 1]), cc, ss);
      v[r] = make_float2(fmaf(v[r].x, cc.x, -v[r].y * ss.x), fmaf(v[r].x, ss.x, v[r].y * cc.x));
      v[r + 1] = make_float2(fmaf(v[r + 1].x, cc.y, -v[r + 1].y * ss.y), fmaf(v[r + 1].x, ss.y, v[r + 1].y * cc.y));
    }
  } else if (__all_sync(0xffffffffu, m <= 0.785398163f)) {
#pragma unroll
    for (int r = 0; r < kFwdR; r += 2) {
      float2 cc, ss;
      expj_pair(make_float2(phi[r], phi[r + 1]), cc, ss);
      v[r] = make_float2(fmaf(v[r].x, cc.x, -v[r].y * ss.x), fmaf(v[r].x, ss.x, v[r].y * cc.x));
      v[r + 1] = make_float2(fmaf(v[r + 1].x, cc.y, -v[r + 1].y * ss.y), fmaf(v[r + 1].x, ss.y, v[r + 1].y * cc.y));
    }
  } else {
#pragma unroll
    for (int r = 0; r < kFwdR; ++r) v[r] = cmul(v[r], expj<true>(phi[r]));
  }
}

}  // namespace ldbp
