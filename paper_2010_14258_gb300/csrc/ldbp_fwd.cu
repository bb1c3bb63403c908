// Fused multi-step learned-DBP forward kernel.
//
// Computes Eq. (7) of the paper with the symmetric circular FIR of Sec. III-B
// as linear step and the Kerr rotation x exp(j c |x|^2) as nonlinear step.
//
// Design (GB300):
//  * One thread block holds a 4096-sample tile: 128 threads x 32 consecutive
//    samples (fixed-width instances and the per-step dispatch up to K = 8) or
//    256 threads x 16 samples (the dispatch for K <= 2 and K <= 16).  The
//    tile covers an output interval of L samples plus the summed overlap-save
//    halo Hp >= sum_i K_i on each side (circular wrap at the waveform ends).
//    It is read from HBM once with a TMA bulk copy (cp.async.bulk, completion
//    on an mbarrier) and written back once with a bulk store: 16 bytes of HBM
//    traffic per sample for all M steps.
//  * The samples live in registers for all M steps.  Neighbour samples for
//    the FIR come from the adjacent lanes by warp shuffles; only the two
//    edge lanes of every warp exchange K samples through shared memory.
//  * The Kerr step evaluates exp(j c |v|^2) with the minimax polynomial tiers
//    of ldbp_tile.cuh (FP32x2 packed, no special-function unit).
//  * The FIR uses the folded form of Fig. 3: y_m = h_0 x_m + sum_k h_k (x_{m-k} + x_{m+k}).
//  * The valid window shrinks by K_i per side per step; after M steps the
//    interior [Hp, Hp + L) of the tile is exact.
#include <cstdio>

#include "common.cuh"
#include "ldbp_fwd.cuh"
#include "ldbp_tile.cuh"

namespace ldbp {

template <int K, int R, int NW>
__device__ __forceinline__ void fir_kerr_step(float2 (&v)[R], const float4* __restrict__ h4, float c,
                                              float2* edge_first, float2* edge_last, int lane, int warp,
                                              bool compute) {
  float2 xe[R + 2 * K];
  tile_extend<K, R, NW>(v, xe, edge_first, edge_last, lane, warp);
  if (!compute) return;
  tile_fir<K, false, R>(xe, h4, v);
  if (c != 0.f) tile_kerr<R>(v, c);
}

template <int KMAX, int R, int NW>
__device__ __forceinline__ void dispatch_step(int K, float2 (&v)[R], const float4* h, float c, float2* ef,
                                              float2* el, int lane, int warp, bool compute) {
  // Every case is a fully unrolled instance; the branch is uniform per block.
  switch (K) {
#define LDBP_CASE(k)                                                    \
  case k:                                                               \
    if constexpr (k <= KMAX) fir_kerr_step<k, R, NW>(v, h, c, ef, el, lane, warp, compute); \
    break;
    LDBP_CASE(0) LDBP_CASE(1) LDBP_CASE(2) LDBP_CASE(3) LDBP_CASE(4) LDBP_CASE(5) LDBP_CASE(6)
    LDBP_CASE(7) LDBP_CASE(8) LDBP_CASE(9) LDBP_CASE(10) LDBP_CASE(11) LDBP_CASE(12) LDBP_CASE(13)
    LDBP_CASE(14) LDBP_CASE(15) LDBP_CASE(16)
#undef LDBP_CASE
    default:
      break;
  }
}

// Loads the S-sample tile starting at circular position g0 of waveform row `src`.
template <int S>
__device__ __forceinline__ void load_tile(float2* tile, const float2* __restrict__ src, long long n, long long g0,
                                          uint64_t* bar, bool* timed_out) {
  const int tid = threadIdx.x;
  const bool contiguous = g0 >= 0 && g0 + S <= n;
  const bool bulk = contiguous && aligned16(src + g0);
  if (bulk) {
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, S * sizeof(float2));
      bulk_g2s(tile, src + g0, S * sizeof(float2), bar);
    }
    if (!mbar_wait_bounded(bar, 0)) *timed_out = true;
  } else {
    for (int s = tid; s < S; s += blockDim.x) {
      long long q = (g0 + s) % n;
      if (q < 0) q += n;
      tile[s] = src[q];
    }
  }
}

// KFIX >= 0: every step has half-width KFIX (compile-time, no per-step dispatch).
// R consecutive samples per thread, NT threads: S = R * NT samples per tile.
template <int KMAX, int MINB, int KFIX, int R = kFwdR, int NT = kFwdNT>
__global__ void __launch_bounds__(NT, MINB) ldbp_fwd_kernel(const __grid_constant__ FwdParams p) {
  constexpr int NW = NT / 32, S = R * NT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);
  float4* taps_s = reinterpret_cast<float4*>(tile + S);        // [M][KMAX+1] (re, re, im, im)
  float2* edges = reinterpret_cast<float2*>(taps_s + p.M * (KMAX + 1));  // [2 parity][2][NW][kFwdEdge]
  uint64_t* bar = reinterpret_cast<uint64_t*>(edges + 4 * NW * kFwdEdge);
  __shared__ bool timed_out;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x / p.tiles_per_wave;
  const int tt = blockIdx.x - b * p.tiles_per_wave;
  const long long n = p.n;
  const long long t0 = (long long)tt * p.L;
  const int Lt = (int)min((long long)p.L, n - t0);
  if (Lt <= 0) return;  // uniform per block
  if (*(volatile int*)&g_device_status == kDevTimeout) return;  // an earlier block gave up waiting
  const float2* src = p.x + (long long)b * n;

  if (tid == 0) {
    timed_out = false;
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int e = tid; e < p.M * (KMAX + 1); e += NT) {
    const int i = e / (KMAX + 1), k = e - i * (KMAX + 1);
    taps_s[e] = tap_pair(k <= p.K[i] ? p.taps[(long long)i * p.taps_stride + k] : make_float2(0.f, 0.f));
  }
  __syncthreads();
  load_tile<S>(tile, src, n, t0 - p.Hp, bar, &timed_out);
  __syncthreads();
  if (timed_out) return;

  // The tile's samples move between shared memory and registers in a
  // swizzled, conflict-free chunk order for the K <= 4 classes (measured 1-4 %
  // faster at T = 3..9); the wider instances keep the plain order (their
  // larger register footprint spilled more with the swizzle: T = 15 1 % slower).
  constexpr bool kSwizzle = KMAX <= 4;
  float2 v[R];
  if constexpr (kSwizzle) {
    load_own_samples<R>(tile, lane, v);
  } else {
    const float4* t4 = reinterpret_cast<const float4*>(tile + tid * R);
#pragma unroll
    for (int r = 0; r < R / 2; ++r) {
      float4 q = t4[r];
      v[2 * r] = make_float2(q.x, q.y);
      v[2 * r + 1] = make_float2(q.z, q.w);
    }
  }
  // Warps entirely beyond the last sample any output depends on skip the arithmetic.
  const bool compute = warp * 32 * R < p.L + 2 * p.Hp;
  const int s0 = tid * R - p.Hp;  // output offset of v[0]

  int parity = 0;
  for (int i = 0; i < p.M; ++i) {
    if (p.ckpt) {
      float2* dst = p.ckpt + ((long long)i * p.batch + b) * n + t0;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (s0 + r >= 0 && s0 + r < Lt) dst[s0 + r] = v[r];
    }
    const int K = p.K[i];
    float2* ef = edges + parity * 2 * NW * kFwdEdge;
    float2* el = ef + NW * kFwdEdge;
    if constexpr (KFIX >= 0)
      fir_kerr_step<KFIX, R, NW>(v, taps_s + i * (KMAX + 1), p.c[i], ef, el, lane, warp, compute);
    else
      dispatch_step<KMAX, R, NW>(K, v, taps_s + i * (KMAX + 1), p.c[i], ef, el, lane, warp, compute);
    if (K > 0) parity ^= 1;
  }

  // Stage the result in shared memory and store the interior once.
  if constexpr (kSwizzle) {
    store_own_samples<R>(tile, lane, v);
  } else {
    float4* t4 = reinterpret_cast<float4*>(tile + tid * R);
#pragma unroll
    for (int r = 0; r < R / 2; ++r) t4[r] = make_float4(v[2 * r].x, v[2 * r].y, v[2 * r + 1].x, v[2 * r + 1].y);
  }
  float2* dst = p.y + (long long)b * n + t0;
  const bool bulk = aligned16(dst) && aligned16(tile + p.Hp) && (Lt % 2 == 0);
  if (bulk) {
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      bulk_s2g(dst, tile + p.Hp, (uint32_t)Lt * sizeof(float2));
      bulk_commit();
      bulk_wait_read0();
    }
  } else {
    __syncthreads();
    for (int s = tid; s < Lt; s += NT) dst[s] = tile[p.Hp + s];
  }
}

size_t fwd_smem_bytes(int kmax, int M, int S) {
  return sizeof(float2) * ((size_t)S + 4 * kFwdNW * kFwdEdge) + sizeof(float4) * (size_t)M * (kmax + 1) + 16;
}

int fwd_kmax_class(int kmax_needed) {
  if (kmax_needed <= 2) return 2;
  if (kmax_needed <= 4) return 4;
  if (kmax_needed <= 8) return 8;
  return 16;
}

template <int KMAX, int MINB, int KFIX, int R = kFwdR, int NT = kFwdNT>
static cudaError_t launch_cls(const FwdParams& p, int grid, cudaStream_t st) {
  const size_t smem = fwd_smem_bytes(KMAX, p.M, R * NT);
  auto kern = ldbp_fwd_kernel<KMAX, MINB, KFIX, R, NT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NT, smem, st>>>(p);
  return cudaGetLastError();
}

// Kernel instance for a model.  Uniform filter widths of the usual models
// (T = 3, 5, 7, 9, 15, 21, 31) get fixed-width instances, mixed widths the per-step
// dispatch.  32 samples per thread in 128-thread blocks except where the
// per-step dispatch over K <= 2 (or up to 16) runs faster with 16 per thread.
enum FwdInstance { kFix1, kFix2, kFix3, kFix4, kFix7, kFix10, kFix15, kGen2, kGen4, kGen8, kGen16 };

static FwdInstance fwd_select(const int* K, int M, int kmax_needed) {
  bool uniform = true;
  for (int i = 1; i < M; ++i) uniform = uniform && K[i] == K[0];
  if (uniform) {
    switch (K[0]) {
      case 1: return kFix1;
      case 2: return kFix2;
      case 3: return kFix3;
      case 4: return kFix4;
      case 7: return kFix7;
      case 10: return kFix10;
      case 15: return kFix15;
      default: break;
    }
  }
  switch (fwd_kmax_class(kmax_needed)) {
    case 2: return kGen2;
    case 4: return kGen4;
    case 8: return kGen8;
    default: return kGen16;
  }
}

int fwd_tile_samples(const int* K, int M, int kmax_needed) {
  switch (fwd_select(K, M, kmax_needed)) {
    case kGen2: case kGen16: return kFwdR * kFwdNT;
    default: return 32 * 128;
  }
}

cudaError_t launch_ldbp_fwd(const FwdParams& p, int kmax_needed, cudaStream_t st) {
  const int grid = p.batch * p.tiles_per_wave;
  switch (fwd_select(p.K, p.M, kmax_needed)) {
    case kFix1: return launch_cls<2, 4, 1, 32, 128>(p, grid, st);
    case kFix2: return launch_cls<2, 4, 2, 32, 128>(p, grid, st);
    case kFix3: return launch_cls<4, 4, 3, 32, 128>(p, grid, st);
    case kFix4: return launch_cls<4, 4, 4, 32, 128>(p, grid, st);
    case kFix7: return launch_cls<8, 3, 7, 32, 128>(p, grid, st);
    case kFix10: return launch_cls<16, 2, 10, 32, 128>(p, grid, st);
    case kFix15: return launch_cls<16, 2, 15, 32, 128>(p, grid, st);
    case kGen2: return launch_cls<2, 3, -1>(p, grid, st);
    case kGen4: return launch_cls<4, 4, -1, 32, 128>(p, grid, st);
    case kGen8: return launch_cls<8, 3, -1, 32, 128>(p, grid, st);
    default: return launch_cls<16, 1, -1>(p, grid, st);
  }
}

}  // namespace ldbp
