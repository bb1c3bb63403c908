// Learned enhanced split-step model (filtered DBP, Sec. III-C, Eqs. (9)-(10)):
// the fused LDBP tile kernel with a filtered power in every nonlinear step,
//   u_{i+1,j} = v_j exp(j c_i sum_{k=-kappa_i}^{kappa_i} eta^(i)_k |v_{j-k}|^2),  v = A_i u_i.
//
// Same tiling as ldbp_fwd_kernel (one 4096-sample tile per block, 16
// consecutive samples per thread in registers, FIR halo by warp shuffles).
// The power |v|^2 of the tile goes to shared memory (double-buffered by step
// parity, so one barrier per step suffices); each thread reads its window of
// 16 + 2 KAPPA powers with 16-byte loads and applies the real filter in
// registers, the taps eta zero-padded to the compile-time KAPPA class (0:
// the power of the sample itself, no shared memory; 8; 20; 24).  The
// phase c * filtered power takes the same minimax polynomial tiers as the
// plain Kerr step.  The halo per side is sum_i (K_i + kappa_i).
#include "ldbp_essm.cuh"

namespace ldbp {

namespace {

// The filtered nonlinear step on the thread's samples: powers to shared
// memory, one barrier, window read, real FIR with zero-padded taps.
template <int KAPPA>
__device__ __forceinline__ void essm_kerr(float2 (&v)[kER], const float* __restrict__ eta_s, float c, float* pbuf,
                                          int tid) {
  constexpr int W = kER + 2 * KAPPA;
  if constexpr (KAPPA == 0) {
    // one tap: the filtered power is eta_0 |v|^2, no neighbour powers needed
    const float e0 = eta_s[0];
    float q[kER];
#pragma unroll
    for (int r = 0; r < kER; ++r) q[r] = e0 * fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
    if (c != 0.f) rotate_by_power(v, q, c);
    return;
  }
  {
    float4* p4 = reinterpret_cast<float4*>(pbuf + ppad(tid * kER));
#pragma unroll
    for (int r = 0; r < kER; r += 4)
      p4[r / 4] = make_float4(fmaf(v[r].x, v[r].x, v[r].y * v[r].y), fmaf(v[r + 1].x, v[r + 1].x, v[r + 1].y * v[r + 1].y),
                              fmaf(v[r + 2].x, v[r + 2].x, v[r + 2].y * v[r + 2].y),
                              fmaf(v[r + 3].x, v[r + 3].x, v[r + 3].y * v[r + 3].y));
  }
  __syncthreads();
  // window [s0 - KAPPA, s0 + kER + KAPPA) of the tile's powers; outside the tile: 0
  float pw[W];
  const int s0 = tid * kER - KAPPA;
  if (s0 >= 0 && s0 + W <= kES && (KAPPA % 4) == 0) {
#pragma unroll
    for (int j = 0; j < W / 4; ++j) {
      const float4 q = *reinterpret_cast<const float4*>(pbuf + ppad(s0 + 4 * j));
      pw[4 * j] = q.x;
      pw[4 * j + 1] = q.y;
      pw[4 * j + 2] = q.z;
      pw[4 * j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < W; ++j) pw[j] = (s0 + j >= 0 && s0 + j < kES) ? pbuf[ppad(s0 + j)] : 0.f;
  }
  float q[kER];
#pragma unroll
  for (int r = 0; r < kER; ++r) q[r] = 0.f;
#pragma unroll
  for (int k = -KAPPA; k <= KAPPA; ++k) {
    const float e = eta_s[k + KAPPA];  // broadcast
#pragma unroll
    for (int r = 0; r < kER; ++r) q[r] = fmaf(e, pw[KAPPA + r - k], q[r]);
  }
  if (c != 0.f) rotate_by_power(v, q, c);
}

template <int K, int KAPPA>
__device__ __forceinline__ void essm_step(float2 (&v)[kER], const float4* __restrict__ h4, const float* eta_s, float c,
                                          float2* ef, float2* el, float* pbuf, int lane, int warp, int tid) {
  float2 xe[kER + 2 * K];
  tile_extend<K, kER, kENW>(v, xe, ef, el, lane, warp);
  tile_fir<K, false, kER>(xe, h4, v);
  essm_kerr<KAPPA>(v, eta_s, c, pbuf, tid);
}

template <int KMAX, int KAPPA>
__device__ __forceinline__ void essm_dispatch(int K, float2 (&v)[kER], const float4* h, const float* eta_s, float c,
                                              float2* ef, float2* el, float* pbuf, int lane, int warp, int tid) {
  switch (K) {
#define LDBP_ECASE(k) \
  case k:             \
    if constexpr (k <= KMAX) essm_step<k, KAPPA>(v, h, eta_s, c, ef, el, pbuf, lane, warp, tid); \
    break;
    LDBP_ECASE(0) LDBP_ECASE(1) LDBP_ECASE(2) LDBP_ECASE(3) LDBP_ECASE(4) LDBP_ECASE(5) LDBP_ECASE(6)
    LDBP_ECASE(7) LDBP_ECASE(8)
#undef LDBP_ECASE
    default:
      break;
  }
}

template <int KMAX, int KAPPA>
__global__ void __launch_bounds__(kENT, 2) ldbp_essm_kernel(const __grid_constant__ EssmParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);
  float* pbufs = reinterpret_cast<float*>(tile + kES);                     // [2][kEPad]
  float4* taps_s = reinterpret_cast<float4*>(pbufs + 2 * kEPad);           // [M][KMAX+1]
  float* eta_s = reinterpret_cast<float*>(taps_s + p.M * (KMAX + 1));      // [M][2 KAPPA + 1], zero-padded
  float2* edges = reinterpret_cast<float2*>(eta_s + ((p.M * (2 * KAPPA + 1) + 3) & ~3));  // [2][2][NW][edge]
  uint64_t* bar = reinterpret_cast<uint64_t*>(edges + 4 * kENW * kFwdEdge);
  __shared__ bool timed_out;
  constexpr int EW = 2 * KAPPA + 1;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x / p.tiles_per_wave;
  const int tt = blockIdx.x - b * p.tiles_per_wave;
  const long long n = p.n;
  const long long t0 = (long long)tt * p.L;
  const int Lt = (int)min((long long)p.L, n - t0);
  if (Lt <= 0) return;
  if (*(volatile int*)&g_device_status == kDevTimeout) return;
  const float2* src = p.x + (long long)b * n;

  if (tid == 0) {
    timed_out = false;
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int e = tid; e < p.M * (KMAX + 1); e += kENT) {
    const int i = e / (KMAX + 1), k = e - i * (KMAX + 1);
    taps_s[e] = tap_pair(k <= p.K[i] ? p.taps[(long long)i * p.taps_stride + k] : make_float2(0.f, 0.f));
  }
  for (int e = tid; e < p.M * EW; e += kENT) {
    const int i = e / EW, k = e - i * EW - KAPPA;  // k in [-KAPPA, KAPPA]
    const int ki = p.kappa[i];
    eta_s[e] = (k >= -ki && k <= ki) ? p.eta[(long long)i * p.eta_stride + k + ki] : 0.f;
  }
  __syncthreads();
  const long long g0 = t0 - p.Hp;
  const bool bulk = g0 >= 0 && g0 + kES <= n && aligned16(src + g0);
  if (bulk) {
    if (tid == 0) {
      mbar_arrive_expect_tx(bar, kES * sizeof(float2));
      bulk_g2s(tile, src + g0, kES * sizeof(float2), bar);
    }
    if (!mbar_wait_bounded(bar, 0)) timed_out = true;
  } else {
    for (int s = tid; s < kES; s += kENT) {
      long long q = (g0 + s) % n;
      if (q < 0) q += n;
      tile[s] = src[q];
    }
  }
  __syncthreads();
  if (timed_out) return;

  float2 v[kER];
  load_own_samples<kER>(tile, lane, v);  // conflict-free swizzled read
  int parity = 0;
  const int s0 = tid * kER - p.Hp;  // output offset of v[0]
  for (int i = 0; i < p.M; ++i) {
    if (p.ckpt) {
      float2* dst = p.ckpt + ((long long)i * p.batch + b) * n + t0;
#pragma unroll
      for (int r = 0; r < kER; ++r)
        if (s0 + r >= 0 && s0 + r < Lt) dst[s0 + r] = v[r];
    }
    float2* ef = edges + parity * 2 * kENW * kFwdEdge;
    float2* el = ef + kENW * kFwdEdge;
    essm_dispatch<KMAX, KAPPA>(p.K[i], v, taps_s + i * (KMAX + 1), eta_s + i * EW, p.c[i], ef, el,
                               pbufs + (i & 1) * kEPad, lane, warp, tid);
    if (p.K[i] > 0) parity ^= 1;
  }

  store_own_samples<kER>(tile, lane, v);
  float2* dst = p.y + (long long)b * n + t0;
  if (aligned16(dst) && aligned16(tile + p.Hp) && (Lt % 2 == 0)) {
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      bulk_s2g(dst, tile + p.Hp, (uint32_t)Lt * sizeof(float2));
      bulk_commit();
      bulk_wait_read0();
    }
  } else {
    __syncthreads();
    for (int s = tid; s < Lt; s += kENT) dst[s] = tile[p.Hp + s];
  }
}

size_t essm_smem_bytes(int kmax, int kappa, int M) {
  return sizeof(float2) * (size_t)kES + sizeof(float) * 2 * (size_t)kEPad + sizeof(float4) * (size_t)M * (kmax + 1) +
         sizeof(float) * (size_t)((M * (2 * kappa + 1) + 3) & ~3) + sizeof(float2) * 4 * kENW * kFwdEdge + 16;
}

template <int KMAX, int KAPPA>
cudaError_t essm_launch(const EssmParams& p, int grid, cudaStream_t st) {
  const size_t smem = essm_smem_bytes(KMAX, KAPPA, p.M);
  auto kern = ldbp_essm_kernel<KMAX, KAPPA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kENT, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace
}  // namespace ldbp

using namespace ldbp;

extern "C" {

int ldbp_essm_apply(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, const float* eta,
                    int32_t eta_stride, const int32_t* kappa, int32_t M, const void* x, void* y, int64_t n,
                    int32_t batch, void* ckpt, void* stream) {
  if (!taps || !T || !c || !eta || !kappa || !x || !y) return fail(LDBP_EINVAL, "pointer arguments must be non-NULL");
  if (n < 1 || batch < 1) return fail(LDBP_EINVAL, "n=%lld, batch=%d must be >= 1", (long long)n, batch);
  int H = 0, hmax = 0, kmax = 0, kapmax = 0;
  if (int rc = essm_check(T, c, kappa, M, taps_stride, eta_stride, &H, &hmax, &kmax, &kapmax)) return rc;
  const size_t bytes = (size_t)n * (size_t)batch * sizeof(float2);
  {
    const char* xb = static_cast<const char*>(x);
    const char* yb = static_cast<const char*>(y);
    if (xb < yb + bytes && yb < xb + bytes) return fail(LDBP_EINVAL, "x and y overlap");
    if (ckpt) {
      const char* cb = static_cast<const char*>(ckpt);
      if ((cb < xb + bytes && xb < cb + bytes * M) || (cb < yb + bytes && yb < cb + bytes * M))
        return fail(LDBP_EINVAL, "ckpt overlaps x or y");
    }
  }
  TilePlan plan;
  if (make_tile_plan(n, H, &plan, kES)) return fail(LDBP_EINVAL, "halo sum %d too large for one tile", H);
  if ((long long)plan.tiles_per_wave * batch > 0x7fffffffLL) return fail(LDBP_EINVAL, "grid too large");
  EssmParams p;
  memset(&p, 0, sizeof(p));
  p.x = static_cast<const float2*>(x);
  p.y = static_cast<float2*>(y);
  p.ckpt = static_cast<float2*>(ckpt);
  p.taps = static_cast<const float2*>(taps);
  p.eta = eta;
  p.taps_stride = taps_stride;
  p.eta_stride = eta_stride;
  p.n = n;
  p.batch = batch;
  p.M = M;
  p.tiles_per_wave = plan.tiles_per_wave;
  p.L = plan.L;
  p.Hp = plan.Hp;
  for (int i = 0; i < M; ++i) {
    p.K[i] = (T[i] - 1) / 2;
    p.kappa[i] = kappa[i];
    p.c[i] = c[i];
  }
  const int grid = batch * plan.tiles_per_wave;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  // filter classes: kappa = 0 (no neighbour powers), <= 8, = 17..20 (the
  // paper's kappa = 20 without the padding of the widest class), <= 24
  if (kmax <= 4)
    e = kapmax == 0   ? essm_launch<4, 0>(p, grid, st)
        : kapmax <= 8 ? essm_launch<4, 8>(p, grid, st)
        : kapmax <= 20 && kapmax > 16 ? essm_launch<4, 20>(p, grid, st)
                      : essm_launch<4, 24>(p, grid, st);
  else
    e = kapmax == 0   ? essm_launch<8, 0>(p, grid, st)
        : kapmax <= 8 ? essm_launch<8, 8>(p, grid, st)
        : kapmax <= 20 && kapmax > 16 ? essm_launch<8, 20>(p, grid, st)
                      : essm_launch<8, 24>(p, grid, st);
  if (e != cudaSuccess) return cuda_fail(e, "ldbp_essm launch");
  return LDBP_OK;
}

}  // extern "C"
