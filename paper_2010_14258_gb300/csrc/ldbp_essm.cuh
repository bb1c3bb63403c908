// Shared parts of the learned enhanced SSM kernels (forward in
// ldbp_essm_fwd.cu, adjoint in ldbp_essm.cu): tile geometry, the parameter
// block of the forward, the rotation by a filtered power and the argument
// checks.  Everything here has internal linkage.
#pragma once

#include <cmath>
#include <cstring>
#include "common.cuh"
#include "ldbp_fwd.cuh"
#include "ldbp_tile.cuh"

namespace ldbp {

namespace {

constexpr int kER = 16, kENT = 256, kENW = kENT / 32, kES = kER * kENT;
// Power buffers are padded by 4 floats per 16: a thread's 16 values start at
// 20 t floats, so 16-byte accesses of 8 consecutive threads hit distinct banks.
constexpr int kEPad = kES + kES / 4;
__device__ __forceinline__ int ppad(int j) { return j + ((j >> 4) << 2); }

struct EssmParams {
  const float2* x;
  float2* y;
  float2* ckpt;      // [M][batch][n] inputs of every step, or nullptr
  const float2* taps;
  const float* eta;  // [M][eta_stride], row i: eta_{-kappa_i} .. eta_{kappa_i}
  int taps_stride, eta_stride;
  long long n;
  int batch, M, tiles_per_wave, L, Hp;
  int K[LDBP_MAX_STEPS];
  int kappa[LDBP_MAX_STEPS];
  float c[LDBP_MAX_STEPS];
};

// v[r] <- v[r] exp(j c q[r]) for a given (filtered) power q; tiers as tile_kerr.
__device__ __forceinline__ void rotate_by_power(float2 (&v)[kER], const float (&q)[kER], float c) {
  float m = 0.f;
#pragma unroll
  for (int r = 0; r < kER; ++r) m = fmaxf(m, fabsf(q[r]));
  m *= fabsf(c);
#define LDBP_ESSM_TIER(fn, k)                                                                               \
  _Pragma("unroll") for (int r = 0; r < kER; r += 2) {                                                      \
    float2 cc, ss;                                                                                          \
    fn(make_float2(q[r], q[r + 1]), k, cc, ss);                                                             \
    v[r] = make_float2(fmaf(v[r].x, cc.x, -v[r].y * ss.x), fmaf(v[r].x, ss.x, v[r].y * cc.x));              \
    v[r + 1] = make_float2(fmaf(v[r + 1].x, cc.y, -v[r + 1].y * ss.y), fmaf(v[r + 1].x, ss.y, v[r + 1].y * cc.y)); \
  }
  if (__all_sync(0xffffffffu, m <= kKerrTierA)) {
    const KerrPolyA k = kerr_poly_a(c);
    LDBP_ESSM_TIER(kerr_pair_a, k)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierB)) {
    const KerrPolyB k = kerr_poly_b(c);
    LDBP_ESSM_TIER(kerr_pair_b, k)
  } else {
#pragma unroll
    for (int r = 0; r < kER; ++r) v[r] = cmul(v[r], expj<true>(c * q[r]));
  }
#undef LDBP_ESSM_TIER
}

// Shared argument checks of the forward and the adjoint: halo H and classes.
int essm_check(const int32_t* T, const float* c, const int32_t* kappa, int32_t M, int32_t taps_stride,
               int32_t eta_stride, int* H, int* hmax, int* kmax, int* kapmax) {
  if (M < 1 || M > LDBP_MAX_STEPS) return fail(LDBP_EINVAL, "M=%d outside 1..%d", M, LDBP_MAX_STEPS);
  if (taps_stride < 1 || eta_stride < 1) return fail(LDBP_EINVAL, "strides must be >= 1");
  *H = *hmax = *kmax = *kapmax = 0;
  for (int i = 0; i < M; ++i) {
    if (T[i] < 1 || T[i] % 2 == 0) return fail(LDBP_EINVAL, "T[%d]=%d must be odd and >= 1", i, T[i]);
    const int K = (T[i] - 1) / 2;
    if (K > LDBP_ESSM_MAX_HALF_TAPS)
      return fail(LDBP_EINVAL, "T[%d]=%d exceeds the supported length %d", i, T[i], 2 * LDBP_ESSM_MAX_HALF_TAPS + 1);
    if (K + 1 > taps_stride) return fail(LDBP_EINVAL, "T[%d]=%d needs taps_stride >= %d", i, T[i], K + 1);
    if (kappa[i] < 0 || kappa[i] > LDBP_ESSM_MAX_KAPPA)
      return fail(LDBP_EINVAL, "kappa[%d]=%d outside 0..%d", i, kappa[i], LDBP_ESSM_MAX_KAPPA);
    if (2 * kappa[i] + 1 > eta_stride)
      return fail(LDBP_EINVAL, "kappa[%d]=%d needs eta_stride >= %d", i, kappa[i], 2 * kappa[i] + 1);
    if (!std::isfinite(c[i])) return fail(LDBP_ENONFINITE, "c[%d] is NaN or infinite", i);
    *H += K + kappa[i];
    *hmax = K + kappa[i] > *hmax ? K + kappa[i] : *hmax;
    *kmax = K > *kmax ? K : *kmax;
    *kapmax = kappa[i] > *kapmax ? kappa[i] : *kapmax;
  }
  return LDBP_OK;
}

}  // namespace
}  // namespace ldbp
