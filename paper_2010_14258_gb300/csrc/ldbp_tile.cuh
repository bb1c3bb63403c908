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
template <int K, int R = kFwdR, int NW = kFwdNW>
__device__ __forceinline__ void tile_extend(const float2 (&v)[R], float2 (&xe)[R + 2 * K], float2* edge_first,
                                            float2* edge_last, int lane, int warp) {
  if constexpr (K > 0) {
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < K; ++j) edge_first[warp * kFwdEdge + j] = v[j];
    }
    if (lane == 31) {
#pragma unroll
      for (int j = 0; j < K; ++j) edge_last[warp * kFwdEdge + j] = v[R - K + j];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      xe[j].x = __shfl_up_sync(0xffffffffu, v[R - K + j].x, 1);
      xe[j].y = __shfl_up_sync(0xffffffffu, v[R - K + j].y, 1);
      xe[K + R + j].x = __shfl_down_sync(0xffffffffu, v[j].x, 1);
      xe[K + R + j].y = __shfl_down_sync(0xffffffffu, v[j].y, 1);
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        xe[j] = warp > 0 ? edge_last[(warp - 1) * kFwdEdge + j] : make_float2(0.f, 0.f);
    }
    if (lane == 31) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        xe[K + R + j] = warp < NW - 1 ? edge_first[(warp + 1) * kFwdEdge + j] : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) xe[K + r] = v[r];
}

// Taps pre-expanded for packed FP32x2 arithmetic: (h.re, h.re, h.im, h.im).
__device__ __forceinline__ float4 tap_pair(float2 h) { return make_float4(h.x, h.x, h.y, h.y); }

// out[r] = h_0 xe[K+r] + sum_k h_k (xe[K+r-k] + xe[K+r+k])   (folded symmetric FIR);
// with CONJ the taps are conjugated (the adjoint filter).  Packed FP32x2
// form: A accumulates h.re * (s.re, s.im) and Bv accumulates h.im * (s.re, s.im),
// so h s = (A.re - Bv.im, A.im + Bv.re): 3 packed instructions per tap pair.
template <int K, bool CONJ, int R = kFwdR>
__device__ __forceinline__ void tile_fir(const float2 (&xe)[R + 2 * K], const float4* __restrict__ h4,
                                         float2 (&out)[R]) {
  float2 hr[K + 1], hi[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) {
    const float4 q = h4[k];
    hr[k] = make_float2(q.x, q.y);
    hi[k] = make_float2(q.z, q.w);
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
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

// Taylor coefficients of sin(c p) and cos(c p) as polynomials in the power
// p = |v|^2 (c folded in): sin = p (s1 + p^2 (s3 + p^2 (s5 + ...))),
// cos = 1 + p^2 (c2 + p^2 (c4 + ...)).  Computed once per step.
struct KerrPoly {
  float s1, s3, s5, s7, s9, c2, c4, c6, c8, c10;
};

__device__ __forceinline__ KerrPoly kerr_poly(float c) {
  KerrPoly k;
  const float c2 = c * c;
  k.s1 = c;
  k.s3 = k.s1 * c2 * -1.66666666666666667e-1f;  // / (2 * 3)
  k.s5 = k.s3 * c2 * -5.0e-2f;                  // / (4 * 5)
  k.s7 = k.s5 * c2 * -2.38095238095238095e-2f;  // / (6 * 7)
  k.s9 = k.s7 * c2 * -1.38888888888888889e-2f;  // / (8 * 9)
  k.c2 = c2 * -0.5f;
  k.c4 = k.c2 * c2 * -8.33333333333333333e-2f;  // / (3 * 4)
  k.c6 = k.c4 * c2 * -3.33333333333333333e-2f;  // / (5 * 6)
  k.c8 = k.c6 * c2 * -1.78571428571428571e-2f;  // / (7 * 8)
  k.c10 = k.c8 * c2 * -1.11111111111111111e-2f; // / (9 * 10)
  return k;
}

// Powers p[r] = |v[r]|^2 of the thread's samples and their maximum.
template <int R = kFwdR>
__device__ __forceinline__ float tile_power(const float2 (&v)[R], float (&p)[R]) {
  float m = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    p[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
    m = fmaxf(m, p[r]);
  }
  return m;
}

// (cos, sin)(c p) for two powers at once, |c p| <= 0.3: series truncated after
// (c p)^5 / (c p)^6 (truncation below 4.4e-8 / 1.7e-9, under half an FP32 ulp of 1).
__device__ __forceinline__ void kerr_pair_small(float2 P, const KerrPoly& k, float2& cs, float2& sn) {
  const float2 r2 = __fmul2_rn(P, P);
  float2 t = __ffma2_rn(r2, make_float2(k.s5, k.s5), make_float2(k.s3, k.s3));
  t = __ffma2_rn(r2, t, make_float2(k.s1, k.s1));
  sn = __fmul2_rn(P, t);
  float2 u = __ffma2_rn(r2, make_float2(k.c6, k.c6), make_float2(k.c4, k.c4));
  u = __ffma2_rn(r2, u, make_float2(k.c2, k.c2));
  cs = __ffma2_rn(r2, u, make_float2(1.f, 1.f));
}

// |c p| <= 0.6: series to (c p)^7 / (c p)^8 (truncation below 2.9e-8 / 1.8e-9).
__device__ __forceinline__ void kerr_pair_mid(float2 P, const KerrPoly& k, float2& cs, float2& sn) {
  const float2 r2 = __fmul2_rn(P, P);
  float2 t = __ffma2_rn(r2, make_float2(k.s7, k.s7), make_float2(k.s5, k.s5));
  t = __ffma2_rn(r2, t, make_float2(k.s3, k.s3));
  t = __ffma2_rn(r2, t, make_float2(k.s1, k.s1));
  sn = __fmul2_rn(P, t);
  float2 u = __ffma2_rn(r2, make_float2(k.c8, k.c8), make_float2(k.c6, k.c6));
  u = __ffma2_rn(r2, u, make_float2(k.c4, k.c4));
  u = __ffma2_rn(r2, u, make_float2(k.c2, k.c2));
  cs = __ffma2_rn(r2, u, make_float2(1.f, 1.f));
}

// The same for |c p| <= pi/4 (series to (c p)^9 / (c p)^10, error below 2e-9).
__device__ __forceinline__ void kerr_pair(float2 P, const KerrPoly& k, float2& cs, float2& sn) {
  const float2 r2 = __fmul2_rn(P, P);
  float2 t = __ffma2_rn(r2, make_float2(k.s9, k.s9), make_float2(k.s7, k.s7));
  t = __ffma2_rn(r2, t, make_float2(k.s5, k.s5));
  t = __ffma2_rn(r2, t, make_float2(k.s3, k.s3));
  t = __ffma2_rn(r2, t, make_float2(k.s1, k.s1));
  sn = __fmul2_rn(P, t);
  float2 u = __ffma2_rn(r2, make_float2(k.c10, k.c10), make_float2(k.c8, k.c8));
  u = __ffma2_rn(r2, u, make_float2(k.c6, k.c6));
  u = __ffma2_rn(r2, u, make_float2(k.c4, k.c4));
  u = __ffma2_rn(r2, u, make_float2(k.c2, k.c2));
  cs = __ffma2_rn(r2, u, make_float2(1.f, 1.f));
}

// Phase tiers of the Kerr step, chosen per warp from its largest phase
// |c p|: the usual per-step nonlinear phase is well below 0.3.
constexpr float kKerrTierA = 0.3f, kKerrTierB = 0.6f, kKerrTierC = 0.785398163f;

// e[r] = exp(j c |v[r]|^2).  Packed FP32x2 Taylor series in p for
// |c p| <= 0.3, 0.6 and pi/4 (tiers A, B, C), the range-reducing scalar path
// (expj) beyond; every path is accurate to about one FP32 ulp.
template <int R = kFwdR>
__device__ __forceinline__ void tile_expj(const float2 (&v)[R], float c, float2 (&e)[R]) {
  float p[R];
  const float m = tile_power(v, p) * fabsf(c);
  const KerrPoly k = kerr_poly(c);
#define LDBP_EXPJ_TIER(fn)                                 \
  _Pragma("unroll") for (int r = 0; r < R; r += 2) {   \
    float2 cc, ss;                                         \
    fn(make_float2(p[r], p[r + 1]), k, cc, ss);            \
    e[r] = make_float2(cc.x, ss.x);                        \
    e[r + 1] = make_float2(cc.y, ss.y);                    \
  }
  if (__all_sync(0xffffffffu, m <= kKerrTierA)) {
    LDBP_EXPJ_TIER(kerr_pair_small)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierB)) {
    LDBP_EXPJ_TIER(kerr_pair_mid)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierC)) {
    LDBP_EXPJ_TIER(kerr_pair)
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) e[r] = expj<true>(c * p[r]);
  }
#undef LDBP_EXPJ_TIER
}

// v[r] <- v[r] exp(j c |v[r]|^2) in place (the Kerr step), without
// materialising the rotation pairs; same tiers as tile_expj.
template <int R = kFwdR>
__device__ __forceinline__ void tile_kerr(float2 (&v)[R], float c) {
  float p[R];
  const float m = tile_power(v, p) * fabsf(c);
  const KerrPoly k = kerr_poly(c);
#define LDBP_KERR_TIER(fn)                                                                                  \
  _Pragma("unroll") for (int r = 0; r < R; r += 2) {                                                    \
    float2 cc, ss;                                                                                          \
    fn(make_float2(p[r], p[r + 1]), k, cc, ss);                                                             \
    v[r] = make_float2(fmaf(v[r].x, cc.x, -v[r].y * ss.x), fmaf(v[r].x, ss.x, v[r].y * cc.x));              \
    v[r + 1] = make_float2(fmaf(v[r + 1].x, cc.y, -v[r + 1].y * ss.y), fmaf(v[r + 1].x, ss.y, v[r + 1].y * cc.y)); \
  }
  if (__all_sync(0xffffffffu, m <= kKerrTierA)) {
    LDBP_KERR_TIER(kerr_pair_small)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierB)) {
    LDBP_KERR_TIER(kerr_pair_mid)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierC)) {
    LDBP_KERR_TIER(kerr_pair)
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cmul(v[r], expj<true>(c * p[r]));
  }
#undef LDBP_KERR_TIER
}

}  // namespace ldbp
