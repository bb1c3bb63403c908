// Adjoint of the fused learned-DBP forward kernel and the deterministic
// reduction of the tap gradients.
//
// Forward step i (Eq. (7), Sec. III-B):  v = A_i u_i (symmetric circular FIR),
// u_{i+1} = v exp(j c_i |v|^2).  With gradients written g = dl/dRe + j dl/dIm:
//   Kerr:  g_v = exp(-j c |v|^2) g_w - 2 c Im(w conj(g_w)) v      (w = u_{i+1})
//   FIR:   g_u = A_i^H g_v  (the same symmetric filter with conjugated taps)
//   taps:  dl/dh_0 = sum_m g_v[m] conj(u[m]),
//          dl/dh_k = sum_m g_v[m] conj(u[m-k] + u[m+k])   (k >= 1).
//   c:     dl/dc = -sum_m |v_m|^2 Im(w_m conj(g_w,m))  (the learnable scaling of
//          the nonlinear step, Remark 1).
// The sweep runs i = M-1 .. 0 inside one kernel.  Each block keeps the
// gradient of its time tile in registers; u_i is re-read per step from the
// step-boundary checkpoints written by ldbp_apply (TMA bulk copies,
// double-buffered two steps ahead) and v is recomputed in the block.  The
// tile halo is H + K_max per side (the adjoint contaminates from the tile
// edges by max(C, K_i) + K_i per step).  Per-block tap sums are written to a
// workspace and summed in a fixed order by ldbp_tap_reduce, so the gradients
// are bitwise reproducible.
#include <cstring>

#include "common.cuh"
#include "ldbp_bwd.cuh"
#include "ldbp_tile.cuh"

namespace ldbp {

struct BwdShared {
  float2* ubuf;    // [2][S]
  float4* taps;    // [M][KMAX+1] (re, re, im, im)
  float2* edges;   // [2 parity][2][NW][kFwdEdge]
  float2* red;     // [NW][KMAX+2]: tap sums, then the c-gradient sum (.x)
  uint64_t* bars;  // [2]
};

// Starts loading u_i (the input of step i) of this block's tile into buffer j.
__device__ __forceinline__ bool issue_ckpt_load(const BwdParams& p, const BwdShared& sh, int j, int i, int b,
                                                long long g0) {
  const long long n = p.n;
  const float2* src = p.ckpt + ((long long)i * p.batch + b) * n;
  float2* dst = sh.ubuf + j * kFwdS;
  const bool bulk = g0 >= 0 && g0 + kFwdS <= n && aligned16(src + g0);
  if (bulk) {
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&sh.bars[j], kFwdS * sizeof(float2));
      bulk_g2s(dst, src + g0, kFwdS * sizeof(float2), &sh.bars[j]);
    }
  } else {
    for (int s = threadIdx.x; s < kFwdS; s += kFwdNT) {
      long long q = (g0 + s) % n;
      if (q < 0) q += n;
      dst[s] = src[q];
    }
  }
  return bulk;
}

template <int K, int KMAX>
__device__ __forceinline__ void bwd_step(int i, float2 (&g)[kFwdR], const float2 (&u)[kFwdR], const BwdParams& p,
                                         const BwdShared& sh, int& parity, int s0, int Lt, int lane, int warp) {
  const float4* h = sh.taps + i * (KMAX + 1);
  const float c = p.c[i];
  float2 xe[kFwdR + 2 * K];
  tile_extend<K>(u, xe, sh.edges + parity * 2 * kFwdNW * kFwdEdge,
                 sh.edges + parity * 2 * kFwdNW * kFwdEdge + kFwdNW * kFwdEdge, lane, warp);
  if (K > 0) parity ^= 1;
  float2 gv[kFwdR];
  float accc = 0.f;  // dl/dc over this thread's own outputs
  if (c != 0.f) {
    float2 v[kFwdR], e[kFwdR];
    tile_fir<K, false>(xe, h, v);
    tile_expj(v, c, e);
#pragma unroll
    for (int r = 0; r < kFwdR; ++r) {
      const float2 w = cmul(e[r], v[r]);  // u_{i+1}
      const float im = fmaf(w.y, g[r].x, -w.x * g[r].y);  // Im(w conj(g))
      const float2 ge = cmulc(g[r], e[r]);                // g conj(e)
      gv[r] = make_float2(fmaf(-2.f * c * im, v[r].x, ge.x), fmaf(-2.f * c * im, v[r].y, ge.y));
      if (s0 + r >= 0 && s0 + r < Lt) accc = fmaf(-fmaf(v[r].x, v[r].x, v[r].y * v[r].y), im, accc);
    }
  } else {
    float2 v[kFwdR];
    tile_fir<K, false>(xe, h, v);  // w = v when c = 0
#pragma unroll
    for (int r = 0; r < kFwdR; ++r) {
      gv[r] = g[r];
      const float im = fmaf(v[r].y, g[r].x, -v[r].x * g[r].y);
      if (s0 + r >= 0 && s0 + r < Lt) accc = fmaf(-fmaf(v[r].x, v[r].x, v[r].y * v[r].y), im, accc);
    }
  }
  // tap gradients over this block's own output interval
  float2 acc[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int r = 0; r < kFwdR; ++r) {
    if (s0 + r >= 0 && s0 + r < Lt) {
      acc[0] = cadd(acc[0], cmulc(gv[r], xe[K + r]));
#pragma unroll
      for (int k = 1; k <= K; ++k) acc[k] = cadd(acc[k], cmulc(gv[r], cadd(xe[K + r - k], xe[K + r + k])));
    }
  }
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
    for (int k = 0; k <= K; ++k) sh.red[warp * (KMAX + 2) + k] = acc[k];
    sh.red[warp * (KMAX + 2) + KMAX + 1] = make_float2(accc, 0.f);
  }
  __syncthreads();
  const int slot = (int)threadIdx.x <= K ? (int)threadIdx.x : (threadIdx.x == KMAX + 1 ? KMAX + 1 : -1);
  if (slot >= 0) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < kFwdNW; ++w) s = cadd(s, sh.red[w * (KMAX + 2) + slot]);
    p.partial[((long long)blockIdx.x * p.M + i) * (KMAX + 2) + slot] = s;
  }
  // g_u = A^H g_v
  float2 ge[kFwdR + 2 * K];
  tile_extend<K>(gv, ge, sh.edges + parity * 2 * kFwdNW * kFwdEdge,
                 sh.edges + parity * 2 * kFwdNW * kFwdEdge + kFwdNW * kFwdEdge, lane, warp);
  if (K > 0) parity ^= 1;
  tile_fir<K, true>(ge, h, g);
}

template <int KMAX>
__device__ __forceinline__ void bwd_dispatch(int K, int i, float2 (&g)[kFwdR], const float2 (&u)[kFwdR],
                                             const BwdParams& p, const BwdShared& sh, int& parity, int s0, int Lt,
                                             int lane, int warp) {
  switch (K) {
#define LDBP_BCASE(k) \
  case k:             \
    if constexpr (k <= KMAX) bwd_step<k, KMAX>(i, g, u, p, sh, parity, s0, Lt, lane, warp); \
    break;
    LDBP_BCASE(0) LDBP_BCASE(1) LDBP_BCASE(2) LDBP_BCASE(3) LDBP_BCASE(4) LDBP_BCASE(5) LDBP_BCASE(6)
    LDBP_BCASE(7) LDBP_BCASE(8) LDBP_BCASE(9) LDBP_BCASE(10) LDBP_BCASE(11) LDBP_BCASE(12) LDBP_BCASE(13)
    LDBP_BCASE(14) LDBP_BCASE(15) LDBP_BCASE(16)
#undef LDBP_BCASE
    default:
      break;
  }
}

template <int KMAX, int MINB>
__global__ void __launch_bounds__(kFwdNT, MINB) ldbp_bwd_kernel(const __grid_constant__ BwdParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  BwdShared sh;
  sh.ubuf = reinterpret_cast<float2*>(smem_raw);
  sh.taps = reinterpret_cast<float4*>(sh.ubuf + 2 * kFwdS);
  sh.edges = reinterpret_cast<float2*>(sh.taps + p.M * (KMAX + 1));
  sh.red = sh.edges + 4 * kFwdNW * kFwdEdge;
  sh.bars = reinterpret_cast<uint64_t*>(sh.red + kFwdNW * (KMAX + 2));
  __shared__ int timed_out;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x / p.tiles_per_wave;
  const int tt = blockIdx.x - b * p.tiles_per_wave;
  const long long n = p.n;
  const long long t0 = (long long)tt * p.L;
  const int Lt = (int)max(0LL, min((long long)p.L, n - t0));
  const long long g0 = t0 - p.Hp;
  const int s0 = tid * kFwdR - p.Hp;

  if (tid == 0) {
    timed_out = 0;
    mbar_init(&sh.bars[0], 1);
    mbar_init(&sh.bars[1], 1);
    fence_mbar_init();
  }
  for (int e = tid; e < p.M * (KMAX + 1); e += kFwdNT) {
    const int i = e / (KMAX + 1), k = e - i * (KMAX + 1);
    sh.taps[e] = tap_pair(k <= p.K[i] ? p.taps[(long long)i * p.taps_stride + k] : make_float2(0.f, 0.f));
  }
  // gradient at the output, straight into registers
  float2 g[kFwdR];
  {
    const float2* src = p.gy + (long long)b * n;
#pragma unroll
    for (int r = 0; r < kFwdR; ++r) {
      long long q = (g0 + tid * kFwdR + r) % n;
      if (q < 0) q += n;
      g[r] = src[q];
    }
  }
  __syncthreads();
  int phase[2] = {0, 0};
  bool bulk[2] = {false, false};
  bulk[(p.M - 1) & 1] = issue_ckpt_load(p, sh, (p.M - 1) & 1, p.M - 1, b, g0);
  if (p.M >= 2) bulk[(p.M - 2) & 1] = issue_ckpt_load(p, sh, (p.M - 2) & 1, p.M - 2, b, g0);

  int parity = 0;
  for (int i = p.M - 1; i >= 0; --i) {
    const int j = i & 1;
    __syncthreads();
    if (bulk[j]) {
      if (!mbar_wait_bounded(&sh.bars[j], phase[j])) timed_out = 1;
      phase[j] ^= 1;
    }
    float2 u[kFwdR];
    load_own_samples<kFwdR>(sh.ubuf + j * kFwdS, lane, u);
    __syncthreads();
    if (timed_out) break;  // uniform: read after the barrier
    if (i >= 2) bulk[j] = issue_ckpt_load(p, sh, j, i - 2, b, g0);
    bwd_dispatch<KMAX>(p.K[i], i, g, u, p, sh, parity, s0, Lt, lane, warp);
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
    for (int r = 0; r < kFwdR; ++r)
      if (s0 + r >= 0 && s0 + r < Lt) dst[s0 + r] = g[r];
  }
}

// gtaps[i][k] = sum over blocks (fixed order, FP64) of the per-block partials;
// zero for k > K_i.  One block per (i, k).
__global__ void __launch_bounds__(256) ldbp_tap_reduce(const float2* __restrict__ partial, int tiles, int M,
                                                       int pstride, const __grid_constant__ TapReduceK kk,
                                                       float2* __restrict__ gtaps, int taps_stride) {
  const int i = blockIdx.x / taps_stride, k = blockIdx.x - i * taps_stride;
  double sx = 0.0, sy = 0.0;
  if (k <= kk.K[i]) {
    for (int t = threadIdx.x; t < tiles; t += 256) {
      const float2 v = partial[((long long)t * M + i) * pstride + k];
      sx += v.x;
      sy += v.y;
    }
  }
  __shared__ double rx[256], ry[256];
  rx[threadIdx.x] = sx;
  ry[threadIdx.x] = sy;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rx[threadIdx.x] += rx[threadIdx.x + o];
      ry[threadIdx.x] += ry[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) gtaps[(long long)i * taps_stride + k] = make_float2((float)rx[0], (float)ry[0]);
}

// gc[i] = sum over blocks (fixed order, FP64) of the c-gradient partials
// (slot pstride - 1, real part).  One block per step.
__global__ void __launch_bounds__(256) ldbp_c_reduce(const float2* __restrict__ partial, int tiles, int M, int pstride,
                                                     float* __restrict__ gc) {
  const int i = blockIdx.x;
  double s = 0.0;
  for (int t = threadIdx.x; t < tiles; t += 256) s += partial[((long long)t * M + i) * pstride + pstride - 1].x;
  __shared__ double r[256];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) r[threadIdx.x] += r[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) gc[i] = (float)r[0];
}

cudaError_t launch_c_reduce(const float2* partial, int tiles, int M, int pstride, float* gc, cudaStream_t st) {
  ldbp_c_reduce<<<M, 256, 0, st>>>(partial, tiles, M, pstride, gc);
  return cudaGetLastError();
}

size_t bwd_smem_bytes(int kmax, int M) {
  return sizeof(float2) * ((size_t)2 * kFwdS + 4 * kFwdNW * kFwdEdge + (size_t)kFwdNW * (kmax + 2)) +
         sizeof(float4) * (size_t)M * (kmax + 1) + 32;
}

template <int KMAX, int MINB>
static cudaError_t launch_bwd_cls(const BwdParams& p, int grid, cudaStream_t st) {
  const size_t smem = bwd_smem_bytes(KMAX, p.M);
  cudaError_t e = cudaFuncSetAttribute(ldbp_bwd_kernel<KMAX, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ldbp_bwd_kernel<KMAX, MINB><<<grid, kFwdNT, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_ldbp_bwd(const BwdParams& p, int kmax_class, cudaStream_t st) {
  const int kf = bwd_fixed_width(p);
  if (kf > 0) return launch_ldbp_bwd_fixed(p, kf, st);
  const int grid = p.batch * p.tiles_per_wave;
  switch (kmax_class) {
    case 2: return launch_bwd_cls<2, 1>(p, grid, st);
    case 4: return launch_bwd_cls<4, 1>(p, grid, st);
    case 8: return launch_bwd_cls<8, 1>(p, grid, st);
    default: return launch_bwd_cls<16, 1>(p, grid, st);
  }
}

cudaError_t launch_tap_reduce(const float2* partial, int tiles, int M, int pstride, const TapReduceK& kk,
                              float2* gtaps, int taps_stride, cudaStream_t st) {
  ldbp_tap_reduce<<<M * taps_stride, 256, 0, st>>>(partial, tiles, M, pstride, kk, gtaps, taps_stride);
  return cudaGetLastError();
}

}  // namespace ldbp
