// Learned-DBP adjoint for every model except mixed-width ones with a filter
// wider than T = 17 (those run ldbp_bwd_kernel): the same reverse sweep and
// the same per-block partial sums as ldbp_bwd_kernel (Eq. (7), Sec. III-B; the
// Kerr and FIR adjoints and the tap and c gradients are stated there),
// computed in a layout that fits two 256-thread blocks per SM up to K = 4
// (one block for the wider classes):
//  * K is a compile-time constant of the step (one instance for a uniform
//    model; a per-step switch over K = 0..8 otherwise);
//  * one pass over sample pairs recomputes the forward FIR output v, applies
//    the Kerr adjoint in place over the incoming gradient and accumulates the
//    tap-gradient products, so v is never held for all samples: the rotation
//    polynomial is chosen per pair (a warp vote) instead of from the largest
//    power of the step; taps and polynomial coefficients are read from
//    shared memory (broadcast);
//  * the tap-gradient products run in packed FP32x2 with two accumulators
//    per tap: P += (g.re s.re, g.im s.im), Q += (g.im s.re, g.re s.im), so that
//    sum g conj(s) = (P.x + P.y, Q.x - Q.y) with no operand swizzle per tap;
//  * each step's checkpoint u_i is read from shared memory in an XOR-swizzled
//    chunk order (no bank conflicts; the per-lane permutation is undone with
//    three stages of selects).
// The partials have the same layout as ldbp_bwd_kernel's ([blocks][M][cls + 2],
// the c-gradient sum in the last slot), so the fixed-order reductions and the
// allocation-free entry point are shared.
#include "common.cuh"
#include "ldbp_bwd.cuh"
#include "ldbp_tile.cuh"

namespace ldbp {

namespace {

constexpr int kR = kFwdR;            // 16 consecutive samples per thread
constexpr int kNT = kFwdNT;          // 256 threads
constexpr int kNW = kNT / 32;
constexpr int kS = kR * kNT;         // 4096-sample tile

struct FixShared {
  float2* ubuf;    // [2][kS] checkpoints (TMA destination, linear)
  float* kerr;     // [M][8] degree-8/7 rotation polynomial of every step (KerrPolyB)
  float4* taps;    // [M][KC+1] (re, re, im, im), zero beyond K_i
  float2* edges;   // [2 parity][2][kNW][kFwdEdge]
  float2* red;     // [kNW][KC+2]
  uint64_t* bars;  // [2]
};

template <int K>
size_t fix_smem_bytes(int M) {
  return sizeof(float2) * ((size_t)2 * kS + 4 * kNW * kFwdEdge + (size_t)kNW * (K + 2)) +
         sizeof(float4) * (size_t)M * (K + 1) + sizeof(float) * 8 * (size_t)M + 32;
}

__device__ __forceinline__ bool fix_issue_load(const BwdParams& p, const FixShared& sh, int j, int i, int b,
                                               long long g0) {
  const long long n = p.n;
  const float2* src = p.ckpt + ((long long)i * p.batch + b) * n;
  float2* dst = sh.ubuf + j * kS;
  const bool bulk = g0 >= 0 && g0 + kS <= n && aligned16(src + g0);
  if (bulk) {
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&sh.bars[j], kS * sizeof(float2));
      bulk_g2s(dst, src + g0, kS * sizeof(float2), &sh.bars[j]);
    }
  } else {
    for (int s = threadIdx.x; s < kS; s += kNT) {
      long long q = (g0 + s) % n;
      if (q < 0) q += n;
      dst[s] = src[q];
    }
  }
  return bulk;
}

// xe = this thread's samples of the tile with K neighbours on each side
// (zeros beyond the tile): own samples from load_own_samples, the lane
// neighbours' by shuffles, and the outer K of lanes 0 and 31 straight from the
// tile.  Reads shared memory only (no barrier; the tile must not change).
template <int K>
__device__ __forceinline__ void extend_from_tile(const float2* tile, int lane, float2 (&xe)[kR + 2 * K]) {
  float2 u[kR];
  load_own_samples(tile, lane, u);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    xe[j].x = __shfl_up_sync(0xffffffffu, u[kR - K + j].x, 1);
    xe[j].y = __shfl_up_sync(0xffffffffu, u[kR - K + j].y, 1);
    xe[K + kR + j].x = __shfl_down_sync(0xffffffffu, u[j].x, 1);
    xe[K + kR + j].y = __shfl_down_sync(0xffffffffu, u[j].y, 1);
  }
  const int base = (int)threadIdx.x * kR;
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int q = base - K + j;
      xe[j] = q >= 0 ? tile[q] : make_float2(0.f, 0.f);
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int q = base + kR + j;
      xe[K + kR + j] = q < kS ? tile[q] : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int r = 0; r < kR; ++r) xe[K + r] = u[r];
}

// One step i of the reverse sweep for a filter of half-width K (taps row h4
// zero-padded to the class width KC): the fused pass over sample pairs, the
// block's tap and c sums (written to the partials), and the conjugate FIR
// g <- A_i^H g_v.  Reads the step's checkpoint tile and, once every thread is
// past the reduction barrier, refills its buffer with step i - 2.
template <int K, int KC>
__device__ __forceinline__ void fix_step(const BwdParams& p, int i, const float2* tile, const float4* h4,
                                         const KerrPolyB* kpoly, float2 (&g)[kR], const FixShared& sh, int& parity,
                                         int lo, int hi, int lane, int warp, int tid, int b, long long g0,
                                         bool& bulk_j) {
  float2* const red = sh.red;
  const float c = p.c[i];
  // One pass over sample pairs: the recomputed forward output v = A_i u
  // (folded FIR, packed), the Kerr adjoint in place over the gradient, and
  // the tap-gradient products dl/dh_k += g_v conj(s_k).  The rotation uses
  // the degree-8/7 polynomials (|c p| <= 1) when every lane's pair is in
  // range, else the range-reducing path, decided per pair and per warp.
  float2 xe[kR + 2 * K];
  extend_from_tile<K>(tile, lane, xe);
  float2 P[K + 1], Q[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) P[k] = Q[k] = make_float2(0.f, 0.f);
  float accc = 0.f;
  const float cabs = fabsf(c);
#pragma unroll
  for (int r = 0; r < kR; r += 2) {
    float2 v[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      const float4 q0 = h4[0];
      float2 A = __fmul2_rn(make_float2(q0.x, q0.y), xe[K + r + d]);
      float2 Bv = __fmul2_rn(make_float2(q0.z, q0.w), xe[K + r + d]);
#pragma unroll
      for (int k = 1; k <= K; ++k) {
        const float4 q = h4[k];
        const float2 sk = __fadd2_rn(xe[K + r + d - k], xe[K + r + d + k]);
        A = __ffma2_rn(make_float2(q.x, q.y), sk, A);
        Bv = __ffma2_rn(make_float2(q.z, q.w), sk, Bv);
      }
      v[d] = __ffma2_rn(make_float2(Bv.y, Bv.x), make_float2(-1.f, 1.f), A);
    }
    const float pw0 = fmaf(v[0].x, v[0].x, v[0].y * v[0].y), pw1 = fmaf(v[1].x, v[1].x, v[1].y * v[1].y);
    if (c != 0.f) {
      float2 e[2];
      if (__all_sync(0xffffffffu, cabs * fmaxf(pw0, pw1) <= kKerrTierB)) {
        const KerrPolyB kb = *kpoly;
        float2 cs, sn;
        kerr_pair_b(make_float2(pw0, pw1), kb, cs, sn);
        e[0] = make_float2(cs.x, sn.x);
        e[1] = make_float2(cs.y, sn.y);
      } else {
        e[0] = expj<true>(c * pw0);
        e[1] = expj<true>(c * pw1);
      }
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const float2 w = cmul(e[d], v[d]);
        const float im = fmaf(w.y, g[r + d].x, -w.x * g[r + d].y);  // Im(w conj(g))
        const float2 ge = cmulc(g[r + d], e[d]);                      // g conj(e)
        const float k2 = -2.f * c * im;
        g[r + d] = make_float2(fmaf(k2, v[d].x, ge.x), fmaf(k2, v[d].y, ge.y));
        if (r + d >= lo && r + d < hi) accc = fmaf(-(d ? pw1 : pw0), im, accc);
      }
    } else {
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const float im = fmaf(v[d].y, g[r + d].x, -v[d].x * g[r + d].y);
        if (r + d >= lo && r + d < hi) accc = fmaf(-(d ? pw1 : pw0), im, accc);
      }
    }
#pragma unroll
    for (int d = 0; d < 2; ++d) {
      if (r + d >= lo && r + d < hi) {
        const float2 g1 = g[r + d], g2 = make_float2(g1.y, g1.x);
        P[0] = __ffma2_rn(g1, xe[K + r + d], P[0]);
        Q[0] = __ffma2_rn(g2, xe[K + r + d], Q[0]);
#pragma unroll
        for (int k = 1; k <= K; ++k) {
          const float2 sk = __fadd2_rn(xe[K + r + d - k], xe[K + r + d + k]);
          P[k] = __ffma2_rn(g1, sk, P[k]);
          Q[k] = __ffma2_rn(g2, sk, Q[k]);
        }
      }
    }
  }
  float2 acc[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) acc[k] = make_float2(P[k].x + P[k].y, Q[k].x - Q[k].y);
#pragma unroll
  for (int k = 0; k <= K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, o);
      acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, o);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) accc += __shfl_xor_sync(0xffffffffu, accc, o);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k <= K; ++k) red[warp * (KC + 2) + k] = acc[k];
    red[warp * (KC + 2) + KC + 1] = make_float2(accc, 0.f);
  }
  __syncthreads();
  // every thread is done reading this step's tile: refill the buffer
  const int j = i & 1;
  if (i >= 2) bulk_j = fix_issue_load(p, sh, j, i - 2, b, g0);
  if (tid <= K || tid == KC + 1) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < kNW; ++w) s = cadd(s, red[w * (KC + 2) + tid]);
    p.partial[((long long)blockIdx.x * p.M + i) * (KC + 2) + tid] = s;
  }
  // g_u = A^H g_v
  float2 ge[kR + 2 * K];
  float2* ef = sh.edges + parity * 2 * kNW * kFwdEdge;
  tile_extend<K, kR, kNW>(g, ge, ef, ef + kNW * kFwdEdge, lane, warp);
  if (K > 0) parity ^= 1;
  tile_fir<K, true, kR>(ge, h4, g);
}

// KFIX >= 0: every step has half-width KFIX; KFIX < 0: per-step dispatch over
// the half-widths 0..KC (uniform per block; KC <= 8).  Two blocks per SM for
// the classes up to K = 4 (128 registers), one for the wider ones.
template <int KC, int KFIX>
__global__ void __launch_bounds__(kNT, (KC <= 4 ? 2 : 1)) ldbp_bwd_fix_kernel(const __grid_constant__ BwdParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FixShared sh;
  sh.ubuf = reinterpret_cast<float2*>(smem_raw);
  sh.taps = reinterpret_cast<float4*>(sh.ubuf + 2 * kS);
  sh.edges = reinterpret_cast<float2*>(sh.taps + p.M * (KC + 1));
  sh.red = sh.edges + 4 * kNW * kFwdEdge;
  sh.bars = reinterpret_cast<uint64_t*>(sh.red + kNW * (KC + 2));
  sh.kerr = reinterpret_cast<float*>(sh.bars + 2);
  __shared__ int timed_out;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x / p.tiles_per_wave;
  const int tt = blockIdx.x - b * p.tiles_per_wave;
  const long long n = p.n;
  const long long t0 = (long long)tt * p.L;
  const int Lt = (int)max(0LL, min((long long)p.L, n - t0));
  const long long g0 = t0 - p.Hp;
  const int s0 = tid * kR - p.Hp;
  // samples r in [lo, hi) of this thread are outputs of this block's interval
  const int lo = max(0, -s0), hi = min(kR, Lt - s0);

  if (tid == 0) {
    timed_out = 0;
    mbar_init(&sh.bars[0], 1);
    mbar_init(&sh.bars[1], 1);
    fence_mbar_init();
  }
  for (int e = tid; e < p.M * (KC + 1); e += kNT) {
    const int i = e / (KC + 1), k = e - i * (KC + 1);
    sh.taps[e] = tap_pair(k <= p.K[i] ? p.taps[(long long)i * p.taps_stride + k] : make_float2(0.f, 0.f));
  }
  for (int i = tid; i < p.M; i += kNT) *reinterpret_cast<KerrPolyB*>(sh.kerr + i * 8) = kerr_poly_b(p.c[i]);
  float2 g[kR];
  {
    const float2* src = p.gy + (long long)b * n;
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      long long q = (g0 + tid * kR + r) % n;
      if (q < 0) q += n;
      g[r] = src[q];
    }
  }
  __syncthreads();
  int phase[2] = {0, 0};
  bool bulk[2] = {false, false};
  bulk[(p.M - 1) & 1] = fix_issue_load(p, sh, (p.M - 1) & 1, p.M - 1, b, g0);
  if (p.M >= 2) bulk[(p.M - 2) & 1] = fix_issue_load(p, sh, (p.M - 2) & 1, p.M - 2, b, g0);

  int parity = 0;
  for (int i = p.M - 1; i >= 0; --i) {
    const int j = i & 1;
    __syncthreads();
    if (bulk[j]) {
      if (!mbar_wait_bounded(&sh.bars[j], phase[j])) timed_out = 1;
      phase[j] ^= 1;
    }
    __syncthreads();
    if (timed_out) break;  // uniform: read after the barrier
    const float2* tile = sh.ubuf + j * kS;
    const float4* h4 = sh.taps + i * (KC + 1);
    const KerrPolyB* kpoly = reinterpret_cast<const KerrPolyB*>(sh.kerr + i * 8);
    bool& bj = bulk[j];
#define LDBP_FIX_STEP(k) fix_step<k, KC>(p, i, tile, h4, kpoly, g, sh, parity, lo, hi, lane, warp, tid, b, g0, bj)
    if constexpr (KFIX >= 0) {
      LDBP_FIX_STEP(KFIX);
    } else {
      switch (p.K[i]) {
        case 0: LDBP_FIX_STEP(0); break;
        case 1: LDBP_FIX_STEP(1); break;
        case 2: LDBP_FIX_STEP(2); break;
        case 3:
          if constexpr (KC >= 3) LDBP_FIX_STEP(3);
          break;
        case 4:
          if constexpr (KC >= 4) LDBP_FIX_STEP(4);
          break;
#define LDBP_FIX_CASE(k) case k: if constexpr (KC >= k) LDBP_FIX_STEP(k); break;
        LDBP_FIX_CASE(5) LDBP_FIX_CASE(6) LDBP_FIX_CASE(7) LDBP_FIX_CASE(8)
#undef LDBP_FIX_CASE
        default: break;
      }
    }
#undef LDBP_FIX_STEP
  }
  if (timed_out) {
    // let in-flight copies land before the block's shared memory is released
    for (int jj = 0; jj < 2; ++jj)
      if (bulk[jj]) mbar_wait_bounded(&sh.bars[jj], phase[jj], 1 << 16);
    return;
  }
  if (p.gx) {
    float2* dst = p.gx + (long long)b * n + t0;
#pragma unroll
    for (int r = 0; r < kR; ++r)
      if (r >= lo && r < hi) dst[s0 + r] = g[r];
  }
}

template <int KC, int KFIX>
cudaError_t launch_fix(const BwdParams& p, int grid, cudaStream_t st) {
  const size_t smem = fix_smem_bytes<KC>(p.M);
  auto kern = ldbp_bwd_fix_kernel<KC, KFIX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kNT, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

int bwd_fixed_width(const BwdParams& p) {
  int kmax = 0;
  bool uniform = true;
  for (int i = 0; i < p.M; ++i) {
    kmax = p.K[i] > kmax ? p.K[i] : kmax;
    uniform = uniform && p.K[i] == p.K[0];
  }
  if (uniform && kmax == 0) return -1;
  const int cls = kmax <= 2 ? 2 : kmax <= 4 ? 4 : kmax <= 8 ? 8 : 16;
  // mixed widths beyond K = 8: the switch over 17 step instances spills
  // heavily at one block per SM; ldbp_bwd_kernel handles those
  if (!uniform && cls == 16) return -1;
  return cls * kFixSel + (uniform ? kmax : kFixMixed);
}

cudaError_t launch_ldbp_bwd_fixed(const BwdParams& p, int sel, cudaStream_t st) {
  const int grid = p.batch * p.tiles_per_wave;
  const int cls = sel / kFixSel, k = sel % kFixSel;
  if (k == kFixMixed) {
    switch (cls) {
      case 2: return launch_fix<2, -1>(p, grid, st);
      case 4: return launch_fix<4, -1>(p, grid, st);
      case 8: return launch_fix<8, -1>(p, grid, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (k) {
#define LDBP_FIX_LAUNCH(kk, cc) case kk: return launch_fix<cc, kk>(p, grid, st);
    LDBP_FIX_LAUNCH(1, 2) LDBP_FIX_LAUNCH(2, 2) LDBP_FIX_LAUNCH(3, 4) LDBP_FIX_LAUNCH(4, 4)
    LDBP_FIX_LAUNCH(5, 8) LDBP_FIX_LAUNCH(6, 8) LDBP_FIX_LAUNCH(7, 8) LDBP_FIX_LAUNCH(8, 8)
    LDBP_FIX_LAUNCH(9, 16) LDBP_FIX_LAUNCH(10, 16) LDBP_FIX_LAUNCH(11, 16) LDBP_FIX_LAUNCH(12, 16)
    LDBP_FIX_LAUNCH(13, 16) LDBP_FIX_LAUNCH(14, 16) LDBP_FIX_LAUNCH(15, 16) LDBP_FIX_LAUNCH(16, 16)
#undef LDBP_FIX_LAUNCH
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ldbp
