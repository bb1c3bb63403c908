// Register-level DFT building blocks (radix 2, 3, 4, 6, 8, 12, 16; W_32 twiddles) and a shared-memory
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

// cos and sin of 2 pi / 16 and 2 pi * 2 / 16, each split into a float head and
// the float rounding of its remainder (head + tail carries about 48 bits).
// The tails matter: the split-step kernel applies the same transform
// thousands of times, and a constant whose float rounding has |w| != 1
// scales every sample passing through it by the same factor each time.
constexpr double kC1d = 0.92387953251128675613, kS1d = 0.38268343236508977173, kR2d = 0.70710678118654752440;
constexpr float kC1h = (float)kC1d, kC1l = (float)(kC1d - (double)kC1h);
constexpr float kS1h = (float)kS1d, kS1l = (float)(kS1d - (double)kS1h);
constexpr float kR2h = (float)kR2d, kR2l = (float)(kR2d - (double)kR2h);
constexpr double kS3d = 0.86602540378443864676;  // sqrt(3) / 2 = sin(2 pi / 6)
constexpr float kS3h = (float)kS3d, kS3l = (float)(kS3d - (double)kS3h);

// c * s for a head/tail constant (c = ch + cl): one rounding of the sum.
__device__ __forceinline__ float mul_hl(float ch, float cl, float v) { return fmaf(ch, v, cl * v); }
// a * c + b * s for head/tail constants c and s.
__device__ __forceinline__ float dot_hl(float a, float ch, float cl, float b, float sh, float sl) {
  return fmaf(a, ch, fmaf(b, sh, fmaf(a, cl, b * sl)));
}

// exp(-j 2 pi e / 16) applied to v; e is a compile-time constant.
template <int e>
__device__ __forceinline__ float2 tw16(float2 v) {
  constexpr int m = e & 15;
  if constexpr (m == 0) return v;
  else if constexpr (m == 4) return make_float2(v.y, -v.x);                 // -j
  else if constexpr (m == 8) return make_float2(-v.x, -v.y);                // -1
  else if constexpr (m == 12) return make_float2(-v.y, v.x);                // +j
  else if constexpr (m == 2) return make_float2(mul_hl(kR2h, kR2l, v.x + v.y), mul_hl(kR2h, kR2l, v.y - v.x));
  else if constexpr (m == 6) return make_float2(mul_hl(kR2h, kR2l, v.y - v.x), -mul_hl(kR2h, kR2l, v.x + v.y));
  else if constexpr (m == 10) return make_float2(-mul_hl(kR2h, kR2l, v.x + v.y), mul_hl(kR2h, kR2l, v.x - v.y));
  else if constexpr (m == 14) return make_float2(mul_hl(kR2h, kR2l, v.x - v.y), mul_hl(kR2h, kR2l, v.x + v.y));
  else {
    // general: v (c - j s) with c = cos(2 pi m / 16), s = sin(2 pi m / 16),
    // both +-cos(pi/8) or +-sin(pi/8) in head/tail form
    constexpr bool c_is_c1 = (m == 1 || m == 15 || m == 7 || m == 9);
    constexpr float csg = (m == 1 || m == 15 || m == 3 || m == 13) ? 1.f : -1.f;
    constexpr float ssg = (m <= 7) ? 1.f : -1.f;
    constexpr float ch = csg * (c_is_c1 ? kC1h : kS1h), cl = csg * (c_is_c1 ? kC1l : kS1l);
    constexpr float sh = ssg * (c_is_c1 ? kS1h : kC1h), sl = ssg * (c_is_c1 ? kS1l : kC1l);
    return make_float2(dot_hl(v.x, ch, cl, v.y, sh, sl), dot_hl(v.y, ch, cl, -v.x, sh, sl));
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

// 3-point DFT on (a0, a1, a2), natural order:
//   X0 = a0 + s,  X1,2 = a0 - s / 2 -+ j (sqrt(3) / 2) (a1 - a2),  s = a1 + a2.
__device__ __forceinline__ void dft3(float2& a0, float2& a1, float2& a2) {
  const float2 s = padd(a1, a2), d = psub(a1, a2);
  const float2 t = __ffma2_rn(s, make_float2(-0.5f, -0.5f), a0);
  // j sqrt(3)/2 d = (-sqrt(3)/2 d.y, sqrt(3)/2 d.x)
  const float2 e = make_float2(-mul_hl(kS3h, kS3l, d.y), mul_hl(kS3h, kS3l, d.x));
  a0 = padd(a0, s);
  a1 = psub(t, e);
  a2 = padd(t, e);
}

// exp(-j 2 pi e / 12) applied to v; e is a compile-time constant.  Every
// value is built from 1/2 (exact) and sqrt(3)/2 (head + tail).
template <int e>
__device__ __forceinline__ float2 tw12(float2 v) {
  constexpr int m = ((e % 12) + 12) % 12;
  if constexpr (m == 0) return v;
  else if constexpr (m == 3) return make_float2(v.y, -v.x);    // -j
  else if constexpr (m == 6) return make_float2(-v.x, -v.y);   // -1
  else if constexpr (m == 9) return make_float2(-v.y, v.x);    // +j
  else {
    // v (c - j s): c = cos(pi m / 6), s = sin(pi m / 6), each 0, +-1/2 or +-sqrt(3)/2
    constexpr bool c_big = (m == 1 || m == 5 || m == 7 || m == 11);  // |c| = sqrt(3)/2, |s| = 1/2
    constexpr float csg = (m == 1 || m == 2 || m == 10 || m == 11) ? 1.f : -1.f;
    constexpr float ssg = (m < 6) ? 1.f : -1.f;
    if constexpr (c_big) {
      // x = c v.x + s v.y, y = c v.y - s v.x with |s| = 1/2 exact
      return make_float2(fmaf(csg * kS3h, v.x, fmaf(csg * kS3l, v.x, 0.5f * ssg * v.y)),
                         fmaf(csg * kS3h, v.y, fmaf(csg * kS3l, v.y, -0.5f * ssg * v.x)));
    } else {
      // |c| = 1/2 exact, |s| = sqrt(3)/2
      return make_float2(fmaf(ssg * kS3h, v.y, fmaf(ssg * kS3l, v.y, 0.5f * csg * v.x)),
                         fmaf(-ssg * kS3h, v.x, fmaf(-ssg * kS3l, v.x, 0.5f * csg * v.y)));
    }
  }
}

template <int R>
__device__ __forceinline__ void dft(float2* a) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2(a[0], a[1]);
  } else if constexpr (R == 3) {
    dft3(a[0], a[1], a[2]);
  } else if constexpr (R == 6) {
    // R1 = 2, R2 = 3: b[m1][k2] = DFT3_{m2} a[m1 + 2 m2]; twiddle W6^{m1 k2} = W12^{2 m1 k2}; DFT2 over m1.
    float2 b0[3] = {a[0], a[2], a[4]};
    float2 b1[3] = {a[1], a[3], a[5]};
    dft3(b0[0], b0[1], b0[2]);
    dft3(b1[0], b1[1], b1[2]);
    b1[1] = tw12<2>(b1[1]);
    b1[2] = tw12<4>(b1[2]);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
      float2 x0 = b0[k2], x1 = b1[k2];
      dft2(x0, x1);
      a[k2] = x0;
      a[k2 + 3] = x1;
    }
  } else if constexpr (R == 12) {
    // R1 = 4, R2 = 3: b[m1][k2] = DFT3_{m2} a[m1 + 4 m2]; twiddle W12^{m1 k2}; DFT4 over m1.
    float2 b[4][3];
#pragma unroll
    for (int m1 = 0; m1 < 4; ++m1) {
      b[m1][0] = a[m1];
      b[m1][1] = a[m1 + 4];
      b[m1][2] = a[m1 + 8];
      dft3(b[m1][0], b[m1][1], b[m1][2]);
    }
    b[1][1] = tw12<1>(b[1][1]);
    b[1][2] = tw12<2>(b[1][2]);
    b[2][1] = tw12<2>(b[2][1]);
    b[2][2] = tw12<4>(b[2][2]);
    b[3][1] = tw12<3>(b[3][1]);
    b[3][2] = tw12<6>(b[3][2]);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
      float2 x0 = b[0][k2], x1 = b[1][k2], x2 = b[2][k2], x3 = b[3][k2];
      dft4(x0, x1, x2, x3);
      a[k2] = x0;
      a[k2 + 3] = x1;
      a[k2 + 6] = x2;
      a[k2 + 9] = x3;
    }
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

// cos(pi k / 16), k = 0..8 (head/tail splits are taken at compile time).
constexpr double kCos16d[9] = {1.0,
                               0.98078528040323044913,
                               0.92387953251128675613,
                               0.83146961230254523708,
                               0.70710678118654752440,
                               0.55557023301960222474,
                               0.38268343236508977173,
                               0.19509032201612826785,
                               0.0};

// exp(-j 2 pi k / 32) applied to v (k compile-time, 0 < k < 16); even k are
// the 16-point constants.
template <int k>
__device__ __forceinline__ float2 tw32(float2 v) {
  if constexpr ((k & 1) == 0) {
    return tw16<k / 2>(v);
  } else {
    static_assert(k > 0 && k < 16, "odd k in 1..15");
    constexpr double c = k <= 8 ? kCos16d[k] : -kCos16d[16 - k];
    constexpr double s = k <= 8 ? kCos16d[8 - k] : kCos16d[k - 8];
    constexpr float ch = (float)c, cl = (float)(c - (double)ch);
    constexpr float sh = (float)s, sl = (float)(s - (double)sh);
    return make_float2(dot_hl(v.x, ch, cl, v.y, sh, sl), dot_hl(v.y, ch, cl, -v.x, sh, sl));
  }
}

template <int k>
__device__ __forceinline__ void tw32_loop(float2* o) {
  if constexpr (k < 16) {
    o[k] = tw32<k>(o[k]);
    tw32_loop<k + 1>(o);
  }
}

// Padded shared-memory index: one spare complex slot every 16 keeps the
// stride-16 scatter of the first Stockham pass free of bank conflicts.
__device__ __forceinline__ int spad(int i) { return i + (i >> 4); }

}  // namespace ldbp
