// Counter-based normal generator for the ASE noise (Philox4x32-10 + Box-Muller).
#pragma once

#include "common.cuh"

namespace ldbp {

// ---------------------------------------------------------------- Philox4x32-10
// Published definition (Salmon et al., SC'11): 10 rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// key bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Complex normal with unit variance per component for ASE bin k (Box-Muller).
__device__ __forceinline__ float2 ase_normal(uint32_t k, uint32_t b, uint32_t span, uint32_t counter, uint32_t seed_lo,
                                             uint32_t seed_hi) {
  const uint4 w = philox4x32_10(make_uint4(k >> 1, b, span, counter), make_uint2(seed_lo, seed_hi));
  const uint32_t wa = (k & 1) ? w.z : w.x;
  const uint32_t wb = (k & 1) ? w.w : w.y;
  const float u1 = fmaf((float)wa, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float u2 = fmaf((float)wb, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
  const float rad = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(rad * c, rad * s);
}

}  // namespace ldbp
