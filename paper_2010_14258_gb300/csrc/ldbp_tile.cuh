// Register-tile helpers shared by the fused learned-DBP kernels: each thread
// holds R consecutive samples (a template parameter, default kFwdR); neighbours
// come from adjacent lanes by warp shuffles and from adjacent warps through a
// small shared-memory edge buffer.
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

__device__ __forceinline__ void swap_if(bool c, float4& a, float4& b) {
  const float4 x = a, y = b;
  a = c ? y : x;
  b = c ? x : y;
}

// u[r] = tile[threadIdx.x * R + r] from shared memory without bank
// conflicts: lane l reads 16-byte chunk q ^ (l & 7) in pass q (eight
// consecutive lanes hit eight different bank groups instead of one), then
// the chunks are swapped back across the bits of l & 7 (three stages of
// selects).  R is a multiple of 16.
template <int R>
__device__ __forceinline__ void load_own_samples(const float2* tile, int lane, float2 (&u)[R]) {
  static_assert(R % 16 == 0, "eight or more 16-byte chunks per thread");
  constexpr int NQ = R / 2;
  const float4* t4 = reinterpret_cast<const float4*>(tile) + threadIdx.x * NQ;
  const int s = lane & 7;
  float4 c[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) c[q] = t4[q ^ s];
  // c[q] holds chunk q ^ s; undo the XOR one bit at a time
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1) {
    const bool sw = (s & bit) != 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if ((q & bit) == 0) swap_if(sw, c[q], c[q | bit]);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    u[2 * q] = make_float2(c[q].x, c[q].y);
    u[2 * q + 1] = make_float2(c[q].z, c[q].w);
  }
}

// tile[threadIdx.x * R + r] = v[r], the inverse of load_own_samples: the
// chunks are permuted first, then pass q writes chunk q ^ (l & 7).
template <int R>
__device__ __forceinline__ void store_own_samples(float2* tile, int lane, const float2 (&v)[R]) {
  static_assert(R % 16 == 0, "eight or more 16-byte chunks per thread");
  constexpr int NQ = R / 2;
  float4* t4 = reinterpret_cast<float4*>(tile) + threadIdx.x * NQ;
  const int s = lane & 7;
  float4 c[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) c[q] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
#pragma unroll
  for (int bit = 1; bit < 8; bit <<= 1) {
    const bool sw = (s & bit) != 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      if ((q & bit) == 0) swap_if(sw, c[q], c[q | bit]);
  }
  // c[q] now holds chunk q ^ s
#pragma unroll
  for (int q = 0; q < NQ; ++q) t4[q ^ s] = c[q];
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
    // (A.re - Bv.im, A.im + Bv.re) as one packed FMA on the swapped Bv (exact: a single rounding per part)
    out[r] = __ffma2_rn(make_float2(Bv.y, Bv.x), CONJ ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f), A);
  }
}

// exp(j phi) for the Kerr step, phi = c p with p = |v|^2, as polynomials in p
// with c folded into the coefficients (computed once per step):
//   sin(phi) = p (s1 + p^2 (s3 + p^2 (s5 + ...))),  cos(phi) = 1 + p^2 (c2 + p^2 (c4 + ...)).
// The coefficients are minimax approximations (Remez exchange, absolute
// error) of sin x by odd and cos x - 1 by even polynomials in x:
//   tier A, |x| <= 0.5: degree 5 / 6, truncation error 2.4e-8 / 8.8e-10;
//   tier B, |x| <= 1.0: degree 7 / 8, truncation error 1.05e-8 / 6.0e-10;
// (paper_2010_14258_gb300/kerr_coeffs.py recomputes them).  With FP32
// evaluation the error stays below one FP32 ulp of 1 (8.6e-8 / 1.2e-7 worst
// case in an exact emulation of the arithmetic below).
constexpr float kKerrTierA = 0.5f, kKerrTierB = 1.0f;
constexpr float kSinA1 = 0.9999996633882672f, kSinA3 = -0.16665588371358184f, kSinA5 = 0.00824692499263815f;
constexpr float kCosA2 = -0.4999999293270643f, kCosA4 = 0.04166494975184432f, kCosA6 = -0.00137702498229312f;
constexpr float kSinB1 = 0.9999999054170744f, kSinB3 = -0.1666654029027963f, kSinB5 = 0.0083287710331470845f,
                kSinB7 = -1.9229923808368593e-4f;
constexpr float kCosB2 = -0.49999998116466243f, kCosB4 = 0.041666483357827591f, kCosB6 = -0.0013883339760550355f,
                kCosB8 = 2.413824676776131e-5f;

struct KerrPolyA {
  float s1, s3, s5, c2, c4, c6;
};
struct KerrPolyB {
  float s1, s3, s5, s7, c2, c4, c6, c8;
};

__device__ __forceinline__ KerrPolyA kerr_poly_a(float c) {
  const float c2 = c * c, c3 = c2 * c, c4 = c2 * c2;
  KerrPolyA k;
  k.s1 = kSinA1 * c;
  k.s3 = kSinA3 * c3;
  k.s5 = kSinA5 * (c4 * c);
  k.c2 = kCosA2 * c2;
  k.c4 = kCosA4 * c4;
  k.c6 = kCosA6 * (c4 * c2);
  return k;
}

__device__ __forceinline__ KerrPolyB kerr_poly_b(float c) {
  const float c2 = c * c, c3 = c2 * c, c4 = c2 * c2, c6 = c4 * c2;
  KerrPolyB k;
  k.s1 = kSinB1 * c;
  k.s3 = kSinB3 * c3;
  k.s5 = kSinB5 * (c4 * c);
  k.s7 = kSinB7 * (c6 * c);
  k.c2 = kCosB2 * c2;
  k.c4 = kCosB4 * c4;
  k.c6 = kCosB6 * c6;
  k.c8 = kCosB8 * (c4 * c4);
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

// (cos, sin)(c p) for two powers at once (packed FP32x2), tier A.
__device__ __forceinline__ void kerr_pair_a(float2 P, const KerrPolyA& k, float2& cs, float2& sn) {
  const float2 r2 = __fmul2_rn(P, P);
  float2 t = __ffma2_rn(r2, make_float2(k.s5, k.s5), make_float2(k.s3, k.s3));
  t = __ffma2_rn(r2, t, make_float2(k.s1, k.s1));
  sn = __fmul2_rn(P, t);
  float2 u = __ffma2_rn(r2, make_float2(k.c6, k.c6), make_float2(k.c4, k.c4));
  u = __ffma2_rn(r2, u, make_float2(k.c2, k.c2));
  cs = __ffma2_rn(r2, u, make_float2(1.f, 1.f));
}

// The same, tier B.
__device__ __forceinline__ void kerr_pair_b(float2 P, const KerrPolyB& k, float2& cs, float2& sn) {
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

// e[r] = exp(j c |v[r]|^2).  The tier is chosen per warp from its largest
// phase |c p|: tier A (the usual per-step nonlinear phase), tier B, and the
// range-reducing scalar path (expj) beyond |c p| = 1.
template <int R = kFwdR>
__device__ __forceinline__ void tile_expj(const float2 (&v)[R], float c, float2 (&e)[R]) {
  float p[R];
  const float m = tile_power(v, p) * fabsf(c);
#define LDBP_EXPJ_TIER(fn, k)                              \
  _Pragma("unroll") for (int r = 0; r < R; r += 2) {       \
    float2 cc, ss;                                         \
    fn(make_float2(p[r], p[r + 1]), k, cc, ss);            \
    e[r] = make_float2(cc.x, ss.x);                        \
    e[r + 1] = make_float2(cc.y, ss.y);                    \
  }
  if (__all_sync(0xffffffffu, m <= kKerrTierA)) {
    const KerrPolyA k = kerr_poly_a(c);
    LDBP_EXPJ_TIER(kerr_pair_a, k)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierB)) {
    const KerrPolyB k = kerr_poly_b(c);
    LDBP_EXPJ_TIER(kerr_pair_b, k)
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
#define LDBP_KERR_TIER(fn, k)                                                                               \
  _Pragma("unroll") for (int r = 0; r < R; r += 2) {                                                        \
    float2 cc, ss;                                                                                          \
    fn(make_float2(p[r], p[r + 1]), k, cc, ss);                                                             \
    v[r] = make_float2(fmaf(v[r].x, cc.x, -v[r].y * ss.x), fmaf(v[r].x, ss.x, v[r].y * cc.x));              \
    v[r + 1] = make_float2(fmaf(v[r + 1].x, cc.y, -v[r + 1].y * ss.y), fmaf(v[r + 1].x, ss.y, v[r + 1].y * cc.y)); \
  }
  if (__all_sync(0xffffffffu, m <= kKerrTierA)) {
    const KerrPolyA k = kerr_poly_a(c);
    LDBP_KERR_TIER(kerr_pair_a, k)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierB)) {
    const KerrPolyB k = kerr_poly_b(c);
    LDBP_KERR_TIER(kerr_pair_b, k)
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = cmul(v[r], expj<true>(c * p[r]));
  }
#undef LDBP_KERR_TIER
}

}  // namespace ldbp
