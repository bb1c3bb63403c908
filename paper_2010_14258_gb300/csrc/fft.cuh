// Register-level DFT building blocks (radix 2, 4, 8, 16) and a shared-memory
// Stockham FFT for the cluster-resident split-step kernel.
//
// Convention: forward DFT X_k = sum_m x_m exp(-j 2 pi k m / N), natural order
// in and out.  The inverse is obtained as conj(DFT(conj(.))) by the caller.
// Radix-R kernels of composite R are built from two smaller DFTs with the
// usual index map m = m1 + R1 m2, k = k2 + R2 k1 (Cooley-Tukey), all
// twiddles being compile-time constants.
#pragma once

#include "common.cuh"

namespace ldbp {

// exp(-j 2 pi e / 16) applied to v; e is a compile-time constant.
template <int e>
__device__ __forceinline__ float2 tw16(float2 v) {
  constexpr int m = e & 15;
  constexpr float C1 = 0.923879532511286756f, S1 = 0.382683432365089772f, R2 = 0.707106781186547524f;
  if constexpr (m == 0) return v;
  else if constexpr (m == 4) return make_float2(v.y, -v.x);                 // -j
  else if constexpr (m == 8) return make_float2(-v.x, -v.y);                // -1
  else if constexpr (m == 12) return make_float2(-v.y, v.x);                // +j
  else if constexpr (m == 2) return make_float2(R2 * (v.x + v.y), R2 * (v.y - v.x));
  else if constexpr (m == 6) return make_float2(R2 * (v.y - v.x), -R2 * (v.x + v.y));
  else if constexpr (m == 10) return make_float2(-R2 * (v.x + v.y), R2 * (v.x - v.y));
  else if constexpr (m == 14) return make_float2(R2 * (v.x - v.y), R2 * (v.x + v.y));
  else {
    // general: (c, -s) with c = cos(2 pi m / 16), s = sin(2 pi m / 16)
    constexpr float c = (m == 1 || m == 15) ? C1 : (m == 3 || m == 13) ? S1 : (m == 5 || m == 11) ? -S1 : -C1;
    constexpr float s = (m == 1 || m == 7) ? S1 : (m == 3 || m == 5) ? C1 : (m == 9 || m == 15) ? -S1 : -C1;
    return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -v.x * s));
  }
}

// Complex add / subtract as one packed FP32x2 instruction each (a - b is
// fma(b, -1, a), exact).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = padd(t, b);
  b = psub(t, b);
}

// 4-point DFT on (a0, a1, a2, a3), natural order.
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3);
  const float2 d = psub(a1, a3);
  const float2 t3 = make_float2(d.y, -d.x);  // -j (a1 - a3)
  a0 = padd(t0, t2);
  a2 = psub(t0, t2);
  a1 = padd(t1, t3);
  a3 = psub(t1, t3);
}

template <int R>
__device__ __forceinline__ void dft(float2* a) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4(a[0], a[1], a[2], a[3]);
  } else if constexpr (R == 8) {
    // R1 = 2, R2 = 4: b[m1][k2] = DFT4_{m2} a[m1 + 2 m2]; twiddle W8^{m1 k2}; DFT2 over m1.
    float2 b0[4] = {a[0], a[2], a[4], a[6]};
    float2 b1[4] = {a[1], a[3], a[5], a[7]};
    dft4(b0[0], b0[1], b0[2], b0[3]);
    dft4(b1[0], b1[1], b1[2], b1[3]);
    b1[1] = tw16<2>(b1[1]);
    b1[2] = tw16<4>(b1[2]);
    b1[3] = tw16<6>(b1[3]);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      float2 x0 = b0[k2], x1 = b1[k2];
      dft2(x0, x1);
      a[k2] = x0;
      a[k2 + 4] = x1;
    }
  } else if constexpr (R == 16) {
    // R1 = R2 = 4: b[m1][k2] = DFT4_{m2} a[m1 + 4 m2]; twiddle W16^{m1 k2}; DFT4 over m1.
    float2 b[4][4];
#pragma unroll
    for (int m1 = 0; m1 < 4; ++m1) {
      b[m1][0] = a[m1];
      b[m1][1] = a[m1 + 4];
      b[m1][2] = a[m1 + 8];
      b[m1][3] = a[m1 + 12];
      dft4(b[m1][0], b[m1][1], b[m1][2], b[m1][3]);
    }
    b[1][1] = tw16<1>(b[1][1]);
    b[1][2] = tw16<2>(b[1][2]);
    b[1][3] = tw16<3>(b[1][3]);
    b[2][1] = tw16<2>(b[2][1]);
    b[2][2] = tw16<4>(b[2][2]);
    b[2][3] = tw16<6>(b[2][3]);
    b[3][1] = tw16<3>(b[3][1]);
    b[3][2] = tw16<6>(b[3][2]);
    b[3][3] = tw16<9>(b[3][3]);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      float2 x0 = b[0][k2], x1 = b[1][k2], x2 = b[2][k2], x3 = b[3][k2];
      dft4(x0, x1, x2, x3);
      a[k2] = x0;
      a[k2 + 4] = x1;
      a[k2 + 8] = x2;
      a[k2 + 12] = x3;
    }
  }
}

// Padded shared-memory index: one spare complex slot every 16 keeps the
// stride-16 scatter of the first Stockham pass free of bank conflicts.
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

}  // namespace ldbp
