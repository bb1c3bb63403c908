// Adjoint of the learned enhanced split-step model (filtered DBP, Sec. III-C,
// Eqs. (9)-(10)); the forward kernel is in ldbp_essm_fwd.cu.
#include "ldbp_essm.cuh"

namespace ldbp {

namespace {

// ---------------------------------------------------------------- adjoint
//
// Reverse sweep (i = M-1 .. 0), per step with v = A_i u_i, p = |v|^2,
// phi = eta * p, w = v e^{j c phi} and g the gradient at w:
//   a = -c Im(w conj(g)),  dl/dp = eta^T * a  (sum_k eta_k a_{m+k}),
//   g_v = e^{-j c phi} g + 2 (dl/dp) v,  dl/deta_k = sum_j a_j p_{j-k},
//   taps as in ldbp_backward, g_u = A_i^H g_v.
// u_i comes from the checkpoints (TMA, double-buffered two steps ahead).
// The tile halo is sum_i (K_i + kappa_i) + max_i (K_i + kappa_i).  Per-block
// sums (taps, then the 2 KAPPA + 1 filter-tap sums) go to the workspace and
// are reduced in a fixed order in FP64.

struct EssmBwdParams {
  const float2* ckpt;
  const float2* gy;
  float2* gx;
  float2* partial;  // [blocks][M][PST], PST = (KMAX + 1) + (2 KAPPA + 1)
  const float2* taps;
  const float* eta;
  int taps_stride, eta_stride;
  long long n;
  int batch, M, tiles_per_wave, L, Hp;
  int K[LDBP_MAX_STEPS];
  int kappa[LDBP_MAX_STEPS];
  float c[LDBP_MAX_STEPS];
};

// e[r] = exp(j c q[r]) for a given (filtered) power q; tiers as tile_expj.
__device__ __forceinline__ void expj_by_power(const float (&q)[kER], float c, float2 (&e)[kER]) {
  float m = 0.f;
#pragma unroll
  for (int r = 0; r < kER; ++r) m = fmaxf(m, fabsf(q[r]));
  m *= fabsf(c);
#define LDBP_ESSM_ETIER(fn, k)                             \
  _Pragma("unroll") for (int r = 0; r < kER; r += 2) {     \
    float2 cc, ss;                                         \
    fn(make_float2(q[r], q[r + 1]), k, cc, ss);            \
    e[r] = make_float2(cc.x, ss.x);                        \
    e[r + 1] = make_float2(cc.y, ss.y);                    \
  }
  if (__all_sync(0xffffffffu, m <= kKerrTierA)) {
    const KerrPolyA k = kerr_poly_a(c);
    LDBP_ESSM_ETIER(kerr_pair_a, k)
  } else if (__all_sync(0xffffffffu, m <= kKerrTierB)) {
    const KerrPolyB k = kerr_poly_b(c);
    LDBP_ESSM_ETIER(kerr_pair_b, k)
  } else {
#pragma unroll
    for (int r = 0; r < kER; ++r) e[r] = expj<true>(c * q[r]);
  }
#undef LDBP_ESSM_ETIER
}

// Reads the window [s0, s0 + W) of a tile-wide shared-memory array (0 outside the tile).
template <int W>
__device__ __forceinline__ void read_window(const float* buf, int s0, float (&out)[W]) {
  if (s0 >= 0 && s0 + W <= kES && (s0 & 3) == 0 && (W & 3) == 0) {
#pragma unroll
    for (int j = 0; j < W / 4; ++j) {
      const float4 q = *reinterpret_cast<const float4*>(buf + ppad(s0 + 4 * j));
      out[4 * j] = q.x;
      out[4 * j + 1] = q.y;
      out[4 * j + 2] = q.z;
      out[4 * j + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < W; ++j) out[j] = (s0 + j >= 0 && s0 + j < kES) ? buf[ppad(s0 + j)] : 0.f;
  }
}

__device__ __forceinline__ void write_tile16(float* buf, int tid, const float (&a)[kER]) {
  float4* p4 = reinterpret_cast<float4*>(buf + ppad(tid * kER));
#pragma unroll
  for (int r = 0; r < kER; r += 4) p4[r / 4] = make_float4(a[r], a[r + 1], a[r + 2], a[r + 3]);
}

struct EssmBwdShared {
  float2* ubuf;   // [2][kES]
  float* pbuf;    // [kEPad]
  float* abuf;    // [kEPad]
  float4* taps;   // [M][KMAX+1]
  float* eta;     // [M][2 KAPPA + 1], zero-padded
  float2* edges;  // [2][2][NW][edge]
  float2* red;    // [NW][PST]
  uint64_t* bars; // [2]
};

template <int KMAX, int KAPPA>
__device__ __forceinline__ void block_sums(const float2* acc, const float* accq, int K, const EssmBwdShared& sh,
                                           const EssmBwdParams& p, int i, int lane, int warp) {
  constexpr int EW = 2 * KAPPA + 1, PST = KMAX + 1 + EW;
  if (lane == 0) {
    for (int k = 0; k <= KMAX; ++k) sh.red[warp * PST + k] = k <= K ? acc[k] : make_float2(0.f, 0.f);
    for (int j = 0; j < EW; ++j) sh.red[warp * PST + KMAX + 1 + j] = make_float2(accq[j], 0.f);
  }
  __syncthreads();
  for (int slot = threadIdx.x; slot < PST; slot += kENT) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < kENW; ++w) s = cadd(s, sh.red[w * PST + slot]);
    p.partial[((long long)blockIdx.x * p.M + i) * PST + slot] = s;
  }
}

template <int K, int KMAX, int KAPPA>
__device__ __forceinline__ void essm_bwd_step(int i, float2 (&g)[kER], const float2 (&u)[kER], const EssmBwdParams& p,
                                              const EssmBwdShared& sh, int& parity, int s0, int Lt, int lane,
                                              int warp) {
  constexpr int EW = 2 * KAPPA + 1, W = kER + 2 * KAPPA;
  const int tid = threadIdx.x;
  const float4* h = sh.taps + i * (KMAX + 1);
  const float* eta = sh.eta + i * EW;
  const float c = p.c[i];
  float2 xe[kER + 2 * K];
  tile_extend<K, kER, kENW>(u, xe, sh.edges + parity * 2 * kENW * kFwdEdge,
                            sh.edges + parity * 2 * kENW * kFwdEdge + kENW * kFwdEdge, lane, warp);
  if (K > 0) parity ^= 1;
  float2 v[kER];
  tile_fir<K, false, kER>(xe, h, v);
  // p = |v|^2 and the filtered power
  float q[kER];
#pragma unroll
  for (int r = 0; r < kER; ++r) q[r] = fmaf(v[r].x, v[r].x, v[r].y * v[r].y);
  write_tile16(sh.pbuf, tid, q);
  __syncthreads();
  float pw[W];
  read_window<W>(sh.pbuf, tid * kER - KAPPA, pw);
#pragma unroll
  for (int r = 0; r < kER; ++r) q[r] = 0.f;
#pragma unroll
  for (int k = -KAPPA; k <= KAPPA; ++k) {
    const float ek = eta[k + KAPPA];
#pragma unroll
    for (int r = 0; r < kER; ++r) q[r] = fmaf(ek, pw[KAPPA + r - k], q[r]);
  }
  float2 e[kER];
  expj_by_power(q, c, e);
  // a = -c Im(w conj(g)), w = e v
  float a[kER];
#pragma unroll
  for (int r = 0; r < kER; ++r) {
    const float2 w = cmul(e[r], v[r]);
    a[r] = -c * fmaf(w.y, g[r].x, -w.x * g[r].y);
  }
  // filter-tap gradient sums over the block's own outputs: sum_j a_j p_{j-k}
  float accq[EW];
#pragma unroll
  for (int j = 0; j < EW; ++j) accq[j] = 0.f;
#pragma unroll
  for (int r = 0; r < kER; ++r) {
    const float ar = (s0 + r >= 0 && s0 + r < Lt) ? a[r] : 0.f;
#pragma unroll
    for (int k = -KAPPA; k <= KAPPA; ++k) accq[k + KAPPA] = fmaf(ar, pw[KAPPA + r - k], accq[k + KAPPA]);
  }
  write_tile16(sh.abuf, tid, a);
  __syncthreads();
  float aw[W];
  read_window<W>(sh.abuf, tid * kER - KAPPA, aw);
  // g_v = conj(e) g + 2 (eta^T * a) v
  float2 gv[kER];
#pragma unroll
  for (int r = 0; r < kER; ++r) {
    float dp = 0.f;
#pragma unroll
    for (int k = -KAPPA; k <= KAPPA; ++k) dp = fmaf(eta[k + KAPPA], aw[KAPPA + r + k], dp);
    const float2 ge = cmulc(g[r], e[r]);
    gv[r] = make_float2(fmaf(2.f * dp, v[r].x, ge.x), fmaf(2.f * dp, v[r].y, ge.y));
  }
  // FIR-tap gradient sums
  float2 acc[K + 1];
#pragma unroll
  for (int k = 0; k <= K; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int r = 0; r < kER; ++r) {
    if (s0 + r >= 0 && s0 + r < Lt) {
      acc[0] = cadd(acc[0], cmulc(gv[r], xe[K + r]));
#pragma unroll
      for (int k = 1; k <= K; ++k) acc[k] = cadd(acc[k], cmulc(gv[r], cadd(xe[K + r - k], xe[K + r + k])));
    }
  }
#pragma unroll
  for (int k = 0; k <= K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, o);
      acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, o);
    }
#pragma unroll
  for (int j = 0; j < EW; ++j)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) accq[j] += __shfl_xor_sync(0xffffffffu, accq[j], o);
  block_sums<KMAX, KAPPA>(acc, accq, K, sh, p, i, lane, warp);
  // g_u = A^H g_v
  float2 ge[kER + 2 * K];
  tile_extend<K, kER, kENW>(gv, ge, sh.edges + parity * 2 * kENW * kFwdEdge,
                            sh.edges + parity * 2 * kENW * kFwdEdge + kENW * kFwdEdge, lane, warp);
  if (K > 0) parity ^= 1;
  tile_fir<K, true, kER>(ge, h, g);
}

template <int KMAX, int KAPPA>
__device__ __forceinline__ void essm_bwd_dispatch(int K, int i, float2 (&g)[kER], const float2 (&u)[kER],
                                                  const EssmBwdParams& p, const EssmBwdShared& sh, int& parity,
                                                  int s0, int Lt, int lane, int warp) {
  switch (K) {
#define LDBP_EBCASE(k) \
  case k:              \
    if constexpr (k <= KMAX) essm_bwd_step<k, KMAX, KAPPA>(i, g, u, p, sh, parity, s0, Lt, lane, warp); \
    break;
    LDBP_EBCASE(0) LDBP_EBCASE(1) LDBP_EBCASE(2) LDBP_EBCASE(3) LDBP_EBCASE(4) LDBP_EBCASE(5) LDBP_EBCASE(6)
    LDBP_EBCASE(7) LDBP_EBCASE(8)
#undef LDBP_EBCASE
    default:
      break;
  }
}

__device__ __forceinline__ bool essm_issue_ckpt(const EssmBwdParams& p, const EssmBwdShared& sh, int j, int i, int b,
                                                long long g0) {
  const long long n = p.n;
  const float2* src = p.ckpt + ((long long)i * p.batch + b) * n;
  float2* dst = sh.ubuf + j * kES;
  const bool bulk = g0 >= 0 && g0 + kES <= n && aligned16(src + g0);
  if (bulk) {
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(&sh.bars[j], kES * sizeof(float2));
      bulk_g2s(dst, src + g0, kES * sizeof(float2), &sh.bars[j]);
    }
  } else {
    for (int s = threadIdx.x; s < kES; s += kENT) {
      long long q = (g0 + s) % n;
      if (q < 0) q += n;
      dst[s] = src[q];
    }
  }
  return bulk;
}

template <int KMAX, int KAPPA>
__global__ void __launch_bounds__(kENT, 1) ldbp_essm_bwd_kernel(const __grid_constant__ EssmBwdParams p) {
  constexpr int EW = 2 * KAPPA + 1, PST = KMAX + 1 + EW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  EssmBwdShared sh;
  sh.ubuf = reinterpret_cast<float2*>(smem_raw);
  sh.pbuf = reinterpret_cast<float*>(sh.ubuf + 2 * kES);
  sh.abuf = sh.pbuf + kEPad;
  sh.taps = reinterpret_cast<float4*>(sh.abuf + kEPad);
  sh.eta = reinterpret_cast<float*>(sh.taps + p.M * (KMAX + 1));
  sh.edges = reinterpret_cast<float2*>(sh.eta + ((p.M * EW + 3) & ~3));
  sh.red = sh.edges + 4 * kENW * kFwdEdge;
  sh.bars = reinterpret_cast<uint64_t*>(sh.red + kENW * PST);
  __shared__ int timed_out;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.x / p.tiles_per_wave;
  const int tt = blockIdx.x - b * p.tiles_per_wave;
  const long long n = p.n;
  const long long t0 = (long long)tt * p.L;
  const int Lt = (int)max(0LL, min((long long)p.L, n - t0));
  const long long g0 = t0 - p.Hp;
  const int s0 = tid * kER - p.Hp;
  if (tid == 0) {
    timed_out = 0;
    mbar_init(&sh.bars[0], 1);
    mbar_init(&sh.bars[1], 1);
    fence_mbar_init();
  }
  for (int e = tid; e < p.M * (KMAX + 1); e += kENT) {
    const int i = e / (KMAX + 1), k = e - i * (KMAX + 1);
    sh.taps[e] = tap_pair(k <= p.K[i] ? p.taps[(long long)i * p.taps_stride + k] : make_float2(0.f, 0.f));
  }
  for (int e = tid; e < p.M * EW; e += kENT) {
    const int i = e / EW, k = e - i * EW - KAPPA;
    const int ki = p.kappa[i];
    sh.eta[e] = (k >= -ki && k <= ki) ? p.eta[(long long)i * p.eta_stride + k + ki] : 0.f;
  }
  float2 g[kER];
  {
    const float2* src = p.gy + (long long)b * n;
#pragma unroll
    for (int r = 0; r < kER; ++r) {
      long long q = (g0 + tid * kER + r) % n;
      if (q < 0) q += n;
      g[r] = src[q];
    }
  }
  __syncthreads();
  int phase[2] = {0, 0};
  bool bulk[2] = {false, false};
  bulk[(p.M - 1) & 1] = essm_issue_ckpt(p, sh, (p.M - 1) & 1, p.M - 1, b, g0);
  if (p.M >= 2) bulk[(p.M - 2) & 1] = essm_issue_ckpt(p, sh, (p.M - 2) & 1, p.M - 2, b, g0);
  int parity = 0;
  for (int i = p.M - 1; i >= 0; --i) {
    const int j = i & 1;
    __syncthreads();
    if (bulk[j]) {
      if (!mbar_wait_bounded(&sh.bars[j], phase[j])) timed_out = 1;
      phase[j] ^= 1;
    }
    float2 u[kER];
    if constexpr (KAPPA <= 8) {
      load_own_samples<kER>(sh.ubuf + j * kES, lane, u);  // conflict-free swizzled read
    } else {
      // the wide-filter classes keep the plain read (the swizzle's registers
      // made them spill more: kappa = 20 8 % slower)
      const float4* t4 = reinterpret_cast<const float4*>(sh.ubuf + j * kES + tid * kER);
#pragma unroll
      for (int r = 0; r < kER / 2; ++r) {
        const float4 q = t4[r];
        u[2 * r] = make_float2(q.x, q.y);
        u[2 * r + 1] = make_float2(q.z, q.w);
      }
    }
    __syncthreads();
    if (timed_out) break;
    if (i >= 2) bulk[j] = essm_issue_ckpt(p, sh, j, i - 2, b, g0);
    essm_bwd_dispatch<KMAX, KAPPA>(p.K[i], i, g, u, p, sh, parity, s0, Lt, lane, warp);
  }
  if (timed_out) {
    for (int jj = 0; jj < 2; ++jj)
      if (bulk[jj]) mbar_wait_bounded(&sh.bars[jj], phase[jj], 1 << 16);
    return;
  }
  if (p.gx) {
    float2* dst = p.gx + (long long)b * n + t0;
#pragma unroll
    for (int r = 0; r < kER; ++r)
      if (s0 + r >= 0 && s0 + r < Lt) dst[s0 + r] = g[r];
  }
}

// gtaps[i][k] (k <= K_i) and geta[i][j] (j < 2 kappa_i + 1) from the per-block
// partials, fixed order, FP64.  One block per output value.
__global__ void __launch_bounds__(256) essm_reduce(const float2* __restrict__ partial, int tiles, int M, int kmax,
                                                   int kappa_cls, const __grid_constant__ EssmBwdParams p,
                                                   float2* __restrict__ gtaps, float* __restrict__ geta) {
  const int pst = kmax + 1 + 2 * kappa_cls + 1;
  const int per = p.taps_stride + p.eta_stride;
  const int i = blockIdx.x / per, o = blockIdx.x - i * per;
  int slot = -1;
  bool is_tap = o < p.taps_stride;
  if (is_tap) {
    if (o <= p.K[i]) slot = o;
  } else {
    const int jj = o - p.taps_stride;
    if (jj < 2 * p.kappa[i] + 1) slot = kmax + 1 + (jj - p.kappa[i] + kappa_cls);
  }
  double sx = 0.0, sy = 0.0;
  if (slot >= 0)
    for (int t = threadIdx.x; t < tiles; t += 256) {
      const float2 v = partial[((long long)t * M + i) * pst + slot];
      sx += v.x;
      sy += v.y;
    }
  __shared__ double rx[256], ry[256];
  rx[threadIdx.x] = sx;
  ry[threadIdx.x] = sy;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rx[threadIdx.x] += rx[threadIdx.x + w];
      ry[threadIdx.x] += ry[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (is_tap)
      gtaps[(long long)i * p.taps_stride + o] = make_float2((float)rx[0], (float)ry[0]);
    else
      geta[(long long)i * p.eta_stride + (o - p.taps_stride)] = (float)rx[0];
  }
}

size_t essm_bwd_smem_bytes(int kmax, int kappa, int M) {
  const int ew = 2 * kappa + 1, pst = kmax + 1 + ew;
  return sizeof(float2) * 2 * (size_t)kES + sizeof(float) * 2 * (size_t)kEPad + sizeof(float4) * (size_t)M * (kmax + 1) +
         sizeof(float) * (size_t)((M * ew + 3) & ~3) + sizeof(float2) * (4 * kENW * kFwdEdge + (size_t)kENW * pst) + 32;
}

template <int KMAX, int KAPPA>
cudaError_t essm_bwd_launch(const EssmBwdParams& p, int grid, float2* gtaps, float* geta, cudaStream_t st) {
  const size_t smem = essm_bwd_smem_bytes(KMAX, KAPPA, p.M);
  auto kern = ldbp_essm_bwd_kernel<KMAX, KAPPA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kENT, smem, st>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  essm_reduce<<<p.M * (p.taps_stride + p.eta_stride), 256, 0, st>>>(p.partial, grid, p.M, KMAX, KAPPA, p, gtaps,
                                                                     geta);
  return cudaGetLastError();
}

}  // namespace
}  // namespace ldbp

using namespace ldbp;

extern "C" {

int ldbp_essm_backward_workspace(int64_t n, int32_t batch, const int32_t* T, const int32_t* kappa, int32_t M,
                                 size_t* bytes) {
  if (!T || !kappa || !bytes) return fail(LDBP_EINVAL, "T, kappa and bytes must be non-NULL");
  if (n < 1 || batch < 1) return fail(LDBP_EINVAL, "n=%lld, batch=%d must be >= 1", (long long)n, batch);
  float zero[LDBP_MAX_STEPS] = {};
  int H = 0, hmax = 0, kmax = 0, kapmax = 0;
  if (int rc = essm_check(T, zero, kappa, M, LDBP_ESSM_MAX_HALF_TAPS + 1, 2 * LDBP_ESSM_MAX_KAPPA + 1, &H, &hmax,
                          &kmax, &kapmax))
    return rc;
  TilePlan plan;
  if (make_tile_plan(n, H + hmax, &plan, kES)) return fail(LDBP_EINVAL, "halo sum too large for one tile");
  const int kcls = kmax <= 4 ? 4 : 8, acls = kapmax <= 8 ? 8 : 24;
  *bytes = (size_t)plan.tiles_per_wave * (size_t)batch * (size_t)M * (size_t)(kcls + 1 + 2 * acls + 1) *
           sizeof(float2);
  return LDBP_OK;
}

int ldbp_essm_backward(const void* taps, int32_t taps_stride, const int32_t* T, const float* c, const float* eta,
                       int32_t eta_stride, const int32_t* kappa, int32_t M, const void* ckpt, const void* gy,
                       void* gx, void* gtaps, float* geta, int64_t n, int32_t batch, void* workspace,
                       size_t workspace_bytes, void* stream) {
  if (!taps || !T || !c || !eta || !kappa || !ckpt || !gy || !gtaps || !geta || !workspace)
    return fail(LDBP_EINVAL, "pointer arguments (except gx) must be non-NULL");
  if (n < 1 || batch < 1) return fail(LDBP_EINVAL, "n=%lld, batch=%d must be >= 1", (long long)n, batch);
  int H = 0, hmax = 0, kmax = 0, kapmax = 0;
  if (int rc = essm_check(T, c, kappa, M, taps_stride, eta_stride, &H, &hmax, &kmax, &kapmax)) return rc;
  size_t need = 0;
  if (int rc = ldbp_essm_backward_workspace(n, batch, T, kappa, M, &need)) return rc;
  if (workspace_bytes < need)
    return fail(LDBP_EINVAL, "workspace of %zu bytes is smaller than the %zu bytes needed", workspace_bytes, need);
  const size_t bytes = (size_t)n * (size_t)batch * sizeof(float2);
  if (gx) {
    const char* xb = static_cast<const char*>(gx);
    const char* gb = static_cast<const char*>(gy);
    const char* cb = static_cast<const char*>(ckpt);
    if ((xb < gb + bytes && gb < xb + bytes) || (xb < cb + bytes * M && cb < xb + bytes))
      return fail(LDBP_EINVAL, "gx overlaps gy or ckpt");
  }
  TilePlan plan;
  make_tile_plan(n, H + hmax, &plan, kES);
  if ((long long)plan.tiles_per_wave * batch > 0x7fffffffLL) return fail(LDBP_EINVAL, "grid too large");
  EssmBwdParams p;
  memset(&p, 0, sizeof(p));
  p.ckpt = static_cast<const float2*>(ckpt);
  p.gy = static_cast<const float2*>(gy);
  p.gx = static_cast<float2*>(gx);
  p.partial = static_cast<float2*>(workspace);
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
  float2* gt = static_cast<float2*>(gtaps);
  cudaError_t e;
  // filter classes: kappa <= 8, exactly 17..20 (the paper's kappa = 20 without
  // padding: smaller windows and fewer sums in registers), else <= 24
  const bool k20 = kapmax >= 17 && kapmax <= 20;
  if (kmax <= 4)
    e = kapmax <= 8 ? essm_bwd_launch<4, 8>(p, grid, gt, geta, st)
        : k20       ? essm_bwd_launch<4, 20>(p, grid, gt, geta, st)
                    : essm_bwd_launch<4, 24>(p, grid, gt, geta, st);
  else
    e = kapmax <= 8 ? essm_bwd_launch<8, 8>(p, grid, gt, geta, st)
        : k20       ? essm_bwd_launch<8, 20>(p, grid, gt, geta, st)
                    : essm_bwd_launch<8, 24>(p, grid, gt, geta, st);
  if (e != cudaSuccess) return cuda_fail(e, "ldbp_essm_backward launch");
  return LDBP_OK;
}

}  // extern "C"
