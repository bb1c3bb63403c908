// Ragged batches of learned-DBP waveforms in one persistent launch.
//
// Waveforms of different length n_w, step count M_w and filter lengths run
// through the same fused tile computation as ldbp_apply (Eq. (7) with the
// FIR of Sec. III-B).  The host builds a work list of (waveform, tile) items
// sorted by decreasing cost (longest-processing-time first); a persistent
// grid (autotuned blocks per SM, up to the occupancy of the K_max class)
// takes items from a device counter until the list is exhausted (no
// spinning: one atomic fetch per item).  The tile
// length per waveform is capped by an autotuned limit that trades halo
// overhead against load balance; the plan can be captured once into a CUDA
// graph (counter reset + launch) and replayed.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "ldbp_fwd.cuh"
#include "ldbp_tile.cuh"

namespace ldbp {

struct RaggedWave {
  long long offset;  // first sample of the waveform in the packed x / y
  long long n;
  int M;
  int step_off;      // first row of the waveform's steps in taps / c / K
  int L;             // output samples per tile
  int Hp;            // halo per side
};

struct RaggedItem {
  int wave;
  int tile;
};

struct RaggedParams {
  const RaggedWave* waves;
  const RaggedItem* items;
  int nitems;
  const int* K;               // [total steps]
  const float* c;             // [total steps]
  const float2* taps;         // [total steps][taps_stride]
  int taps_stride;
  const float2* x;
  float2* y;
  int* counter;
  unsigned long long* done_ns;   // [waves] completion time, or nullptr
  unsigned long long* start_ns;  // [1] earliest block start, or nullptr
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int KMAX, int R, int NW>
__device__ __forceinline__ void ragged_step(int K, float2 (&v)[R], const float4* h, float c, float2* ef,
                                            float2* el, int lane, int warp, bool compute) {
  switch (K) {
#define LDBP_RCASE(k)                                                        \
  case k:                                                                    \
    if constexpr (k <= KMAX) {                                               \
      float2 xe[R + 2 * k];                                                  \
      tile_extend<k, R, NW>(v, xe, ef, el, lane, warp);                      \
      if (compute) {                                                         \
        tile_fir<k, false, R>(xe, h, v);                                     \
        if (c != 0.f) tile_kerr<R>(v, c);                                    \
      }                                                                      \
    }                                                                        \
    break;
    LDBP_RCASE(0) LDBP_RCASE(1) LDBP_RCASE(2) LDBP_RCASE(3) LDBP_RCASE(4) LDBP_RCASE(5) LDBP_RCASE(6)
    LDBP_RCASE(7) LDBP_RCASE(8) LDBP_RCASE(9) LDBP_RCASE(10) LDBP_RCASE(11) LDBP_RCASE(12) LDBP_RCASE(13)
    LDBP_RCASE(14) LDBP_RCASE(15) LDBP_RCASE(16)
#undef LDBP_RCASE
    default:
      break;
  }
}

// R consecutive samples per thread, NT threads (R * NT = kFwdS samples per tile).
template <int KMAX, int R, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) ldbp_ragged_kernel(const __grid_constant__ RaggedParams p) {
  static_assert(R * NT == kFwdS, "tile size");
  constexpr int NW = NT / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);
  float4* taps_s = reinterpret_cast<float4*>(tile + kFwdS);          // [LDBP_MAX_STEPS][KMAX+1]
  float2* edges = reinterpret_cast<float2*>(taps_s + LDBP_MAX_STEPS * (KMAX + 1));  // [2][2][NW][edge]
  uint64_t* bar = reinterpret_cast<uint64_t*>(edges + 4 * NW * kFwdEdge);
  __shared__ int item_s, K_s[LDBP_MAX_STEPS];
  __shared__ float c_s[LDBP_MAX_STEPS];
  __shared__ int timed_out;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    timed_out = 0;
    mbar_init(bar, 1);
    fence_mbar_init();
    if (p.start_ns) atomicMin(p.start_ns, global_ns());
  }
  uint32_t phase = 0;
  int parity = 0;
  for (;;) {
    __syncthreads();  // previous item fully stored; shared buffers free
    if (tid == 0) item_s = atomicAdd(p.counter, 1);
    __syncthreads();
    const int it = item_s;
    if (it >= p.nitems || timed_out) break;
    const RaggedItem item = p.items[it];
    const RaggedWave w = p.waves[item.wave];
    const long long n = w.n, t0 = (long long)item.tile * w.L;
    const int Lt = (int)min((long long)w.L, n - t0);
    for (int i = tid; i < w.M; i += NT) {
      K_s[i] = p.K[w.step_off + i];
      c_s[i] = p.c[w.step_off + i];
    }
    __syncthreads();
    for (int e = tid; e < w.M * (KMAX + 1); e += NT) {
      const int i = e / (KMAX + 1), k = e - i * (KMAX + 1);
      taps_s[e] = tap_pair(k <= K_s[i] ? p.taps[(long long)(w.step_off + i) * p.taps_stride + k]
                                       : make_float2(0.f, 0.f));
    }
    // tile load (TMA bulk copy when contiguous and aligned, else circular plain loads)
    const float2* src = p.x + w.offset;
    const long long g0 = t0 - w.Hp;
    const bool bulk_in = g0 >= 0 && g0 + kFwdS <= n && aligned16(src + g0);
    if (bulk_in) {
      if (tid == 0) {
        mbar_arrive_expect_tx(bar, kFwdS * sizeof(float2));
        bulk_g2s(tile, src + g0, kFwdS * sizeof(float2), bar);
      }
      if (!mbar_wait_bounded(bar, phase)) timed_out = 1;
      phase ^= 1;
    } else {
      for (int s = tid; s < kFwdS; s += NT) {
        long long q = (g0 + s) % n;
        if (q < 0) q += n;
        tile[s] = src[q];
      }
    }
    __syncthreads();
    if (timed_out) break;
    float2 v[R];
    {
      const float4* t4 = reinterpret_cast<const float4*>(tile + tid * R);
#pragma unroll
      for (int r = 0; r < R / 2; ++r) {
        const float4 q = t4[r];
        v[2 * r] = make_float2(q.x, q.y);
        v[2 * r + 1] = make_float2(q.z, q.w);
      }
    }
    const bool compute = warp * 32 * R < w.L + 2 * w.Hp;
    for (int i = 0; i < w.M; ++i) {
      const int K = K_s[i];
      float2* ef = edges + parity * 2 * NW * kFwdEdge;
      ragged_step<KMAX, R, NW>(K, v, taps_s + i * (KMAX + 1), c_s[i], ef, ef + NW * kFwdEdge, lane, warp, compute);
      if (K > 0) parity ^= 1;
    }
    {
      float4* t4 = reinterpret_cast<float4*>(tile + tid * R);
#pragma unroll
      for (int r = 0; r < R / 2; ++r)
        t4[r] = make_float4(v[2 * r].x, v[2 * r].y, v[2 * r + 1].x, v[2 * r + 1].y);
    }
    float2* dst = p.y + w.offset + t0;
    const bool bulk_out = aligned16(dst) && aligned16(tile + w.Hp) && (Lt % 2 == 0);
    if (bulk_out) {
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        bulk_s2g(dst, tile + w.Hp, (uint32_t)Lt * sizeof(float2));
        bulk_commit();
        bulk_wait0();  // the tile buffer is reused by the next item; the store is complete before the timestamp
      }
    } else {
      __syncthreads();
      for (int s = tid; s < Lt; s += NT) dst[s] = tile[w.Hp + s];
      __syncthreads();
    }
    if (tid == 0 && p.done_ns) {
      __threadfence();
      atomicMax(&p.done_ns[item.wave], global_ns());
    }
  }
}

size_t ragged_smem_bytes(int kmax) {
  return sizeof(float2) * ((size_t)kFwdS + 4 * kFwdNW * kFwdEdge) +
         sizeof(float4) * (size_t)LDBP_MAX_STEPS * (kmax + 1) + 16;
}

// Kernel geometry per K_max class: 32 samples per thread in 128-thread blocks,
// except K <= 2 (16 per thread, 256 threads), as for ldbp_apply's dispatch.
template <int KMAX> struct RaggedGeom { static constexpr int R = 32, NT = 128, MINB = KMAX <= 4 ? 4 : KMAX <= 8 ? 3 : 2; };
template <> struct RaggedGeom<2> { static constexpr int R = kFwdR, NT = kFwdNT, MINB = 2; };

template <int KMAX>
static cudaError_t ragged_prepare(int* blocks_per_sm) {
  using G = RaggedGeom<KMAX>;
  auto kern = ldbp_ragged_kernel<KMAX, G::R, G::NT, G::MINB>;
  const size_t smem = ragged_smem_bytes(KMAX);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kern, G::NT, smem);
}

template <int KMAX>
static cudaError_t ragged_launch(const RaggedParams& p, int grid, cudaStream_t st) {
  using G = RaggedGeom<KMAX>;
  ldbp_ragged_kernel<KMAX, G::R, G::NT, G::MINB><<<grid, G::NT, ragged_smem_bytes(KMAX), st>>>(p);
  return cudaGetLastError();
}

struct RaggedPlan {
  int count = 0, kmax_class = 2, total_steps = 0, taps_stride = 0;
  std::vector<long long> n, offset;
  std::vector<int> M, step_off, Kst, H;
  long long total_samples = 0;
  int tile_cap = kFwdS;       // autotuned upper bound on the output samples per tile
  int grid_mult = 1;          // autotuned blocks per SM (bounded by occupancy)
  int max_blocks_per_sm = 1, sm_count = 0, device = 0;
  RaggedWave* d_waves = nullptr;
  RaggedItem* d_items = nullptr;
  int* d_K = nullptr;
  int* d_counter = nullptr;
  int nitems = 0;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;
};

static cudaError_t ragged_build_items(RaggedPlan& pl) {
  std::vector<RaggedWave> waves((size_t)pl.count);
  std::vector<std::pair<double, RaggedItem>> items;
  for (int w = 0; w < pl.count; ++w) {
    TilePlan tp;
    make_tile_plan(pl.n[w], pl.H[w], &tp);
    // cap the tile length: more, shorter tiles balance the persistent grid better
    int L = tp.L;
    long long tpw = tp.tiles_per_wave;
    if (L > pl.tile_cap) {
      tpw = (pl.n[w] + pl.tile_cap - 1) / pl.tile_cap;
      L = (int)((pl.n[w] + tpw - 1) / tpw);
      L += L & 1;
    }
    waves[w] = {pl.offset[w], pl.n[w], pl.M[w], pl.step_off[w], L, tp.Hp};
    double cost = 0;
    for (int i = 0; i < pl.M[w]; ++i) cost += 6.0 * pl.Kst[pl.step_off[w] + i] + 20.0;
    for (long long t = 0; t < tpw; ++t) items.push_back({cost, RaggedItem{w, (int)t}});
  }
  std::stable_sort(items.begin(), items.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  std::vector<RaggedItem> flat(items.size());
  for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].second;
  if (pl.d_items) cudaFree(pl.d_items);
  if (pl.d_waves) cudaFree(pl.d_waves);
  cudaError_t e = cudaMalloc(&pl.d_waves, waves.size() * sizeof(RaggedWave));
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(pl.d_waves, waves.data(), waves.size() * sizeof(RaggedWave), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&pl.d_items, flat.size() * sizeof(RaggedItem));
  if (e != cudaSuccess) return e;
  pl.nitems = (int)flat.size();
  return cudaMemcpy(pl.d_items, flat.data(), flat.size() * sizeof(RaggedItem), cudaMemcpyHostToDevice);
}

static int ragged_enqueue(RaggedPlan& pl, const void* taps, const float* c, const void* x, void* y,
                          unsigned long long* done_ns, unsigned long long* start_ns, cudaStream_t st) {
  RaggedParams p;
  memset(&p, 0, sizeof(p));
  p.waves = pl.d_waves;
  p.items = pl.d_items;
  p.nitems = pl.nitems;
  p.K = pl.d_K;
  p.c = c;
  p.taps = static_cast<const float2*>(taps);
  p.taps_stride = pl.taps_stride;
  p.x = static_cast<const float2*>(x);
  p.y = static_cast<float2*>(y);
  p.counter = pl.d_counter;
  p.done_ns = done_ns;
  p.start_ns = start_ns;
  LDBP_CUDA_TRY(cudaMemsetAsync(pl.d_counter, 0, sizeof(int), st));
  const int grid = pl.sm_count * std::min(pl.grid_mult, pl.max_blocks_per_sm);
  cudaError_t e;
  switch (pl.kmax_class) {
    case 2: e = ragged_launch<2>(p, grid, st); break;
    case 4: e = ragged_launch<4>(p, grid, st); break;
    case 8: e = ragged_launch<8>(p, grid, st); break;
    default: e = ragged_launch<16>(p, grid, st); break;
  }
  if (e != cudaSuccess) return cuda_fail(e, "ragged launch");
  return LDBP_OK;
}

static void ragged_free(RaggedPlan* pl) {
  if (pl->graph) cudaGraphExecDestroy(pl->graph);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  if (pl->d_waves) cudaFree(pl->d_waves);
  if (pl->d_items) cudaFree(pl->d_items);
  if (pl->d_K) cudaFree(pl->d_K);
  if (pl->d_counter) cudaFree(pl->d_counter);
  delete pl;
}

}  // namespace ldbp

using namespace ldbp;

extern "C" {

int ldbp_ragged_plan_create(void** plan, int32_t count, const int64_t* n, const int32_t* M, const int32_t* T,
                            int32_t taps_stride) {
  if (!plan || !n || !M || !T) return fail(LDBP_EINVAL, "plan, n, M and T must be non-NULL");
  if (count < 1) return fail(LDBP_EINVAL, "count=%d must be >= 1", count);
  if (taps_stride < 1) return fail(LDBP_EINVAL, "taps_stride must be >= 1");
  RaggedPlan* pl = new RaggedPlan();
  pl->count = count;
  pl->taps_stride = taps_stride;
  int kmax = 0, so = 0;
  long long off = 0;
  for (int w = 0; w < count; ++w) {
    if (n[w] < 1 || M[w] < 1 || M[w] > LDBP_MAX_STEPS) {
      delete pl;
      return fail(LDBP_EINVAL, "waveform %d: n=%lld, M=%d out of range", w, (long long)n[w], M[w]);
    }
    int H = 0;
    for (int i = 0; i < M[w]; ++i) {
      const int t = T[so + i];
      if (t < 1 || t % 2 == 0 || (t - 1) / 2 > LDBP_MAX_HALF_TAPS || (t - 1) / 2 + 1 > taps_stride) {
        delete pl;
        return fail(LDBP_EINVAL, "waveform %d step %d: T=%d invalid for taps_stride %d", w, i, t, taps_stride);
      }
      const int K = (t - 1) / 2;
      pl->Kst.push_back(K);
      H += K;
      kmax = std::max(kmax, K);
    }
    TilePlan tp;
    if (make_tile_plan(n[w], H, &tp)) {
      delete pl;
      return fail(LDBP_EINVAL, "waveform %d: halo sum %d too large for one tile", w, H);
    }
    pl->n.push_back(n[w]);
    pl->M.push_back(M[w]);
    pl->step_off.push_back(so);
    pl->offset.push_back(off);
    pl->H.push_back(H);
    so += M[w];
    off += n[w];
  }
  pl->total_steps = so;
  pl->total_samples = off;
  pl->kmax_class = fwd_kmax_class(kmax);
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device);
  if (e == cudaSuccess) {
    switch (pl->kmax_class) {
      case 2: e = ragged_prepare<2>(&pl->max_blocks_per_sm); break;
      case 4: e = ragged_prepare<4>(&pl->max_blocks_per_sm); break;
      case 8: e = ragged_prepare<8>(&pl->max_blocks_per_sm); break;
      default: e = ragged_prepare<16>(&pl->max_blocks_per_sm); break;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_K, pl->Kst.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(pl->d_K, pl->Kst.data(), pl->Kst.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&pl->d_counter, sizeof(int));
  if (e == cudaSuccess) {
    pl->max_blocks_per_sm = std::max(1, pl->max_blocks_per_sm);
    pl->grid_mult = pl->max_blocks_per_sm;
    e = ragged_build_items(*pl);
  }
  if (e != cudaSuccess) {
    ragged_free(pl);
    return cuda_fail(e, "ragged plan");
  }
  *plan = pl;
  return LDBP_OK;
}

int ldbp_ragged_plan_destroy(void* plan) {
  if (!plan) return fail(LDBP_EINVAL, "plan must be non-NULL");
  ragged_free(static_cast<RaggedPlan*>(plan));
  return LDBP_OK;
}

int ldbp_ragged_info(const void* plan, int64_t* total_samples, int32_t* total_steps, int32_t* items,
                     int32_t* tile_cap, int32_t* blocks_per_sm) {
  if (!plan) return fail(LDBP_EINVAL, "plan must be non-NULL");
  const RaggedPlan* pl = static_cast<const RaggedPlan*>(plan);
  if (total_samples) *total_samples = pl->total_samples;
  if (total_steps) *total_steps = pl->total_steps;
  if (items) *items = pl->nitems;
  if (tile_cap) *tile_cap = pl->tile_cap;
  if (blocks_per_sm) *blocks_per_sm = std::min(pl->grid_mult, pl->max_blocks_per_sm);
  return LDBP_OK;
}

int ldbp_apply_ragged(void* plan, const void* taps, const float* c, const void* x, void* y, uint64_t* done_ns,
                      uint64_t* start_ns, void* stream) {
  if (!plan || !taps || !c || !x || !y) return fail(LDBP_EINVAL, "plan, taps, c, x and y must be non-NULL");
  RaggedPlan* pl = static_cast<RaggedPlan*>(plan);
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != pl->device) return fail(LDBP_EINVAL, "plan belongs to device %d, current device is %d", pl->device, dev);
  const char* xb = static_cast<const char*>(x);
  const char* yb = static_cast<const char*>(y);
  const size_t bytes = (size_t)pl->total_samples * sizeof(float2);
  if (xb < yb + bytes && yb < xb + bytes) return fail(LDBP_EINVAL, "x and y overlap");
  return ragged_enqueue(*pl, taps, c, x, y, reinterpret_cast<unsigned long long*>(done_ns),
                        reinterpret_cast<unsigned long long*>(start_ns), static_cast<cudaStream_t>(stream));
}

int ldbp_ragged_autotune(void* plan, const void* taps, const float* c, const void* x, void* y, void* stream) {
  if (!plan) return fail(LDBP_EINVAL, "plan must be non-NULL");
  RaggedPlan* pl = static_cast<RaggedPlan*>(plan);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int caps[] = {kFwdS, 3072, 2048, 1024};
  float best = 1e30f;
  int best_cap = pl->tile_cap, best_mult = pl->grid_mult;
  cudaEvent_t e0, e1;
  LDBP_CUDA_TRY(cudaEventCreate(&e0));
  LDBP_CUDA_TRY(cudaEventCreate(&e1));
  for (int cap : caps) {
    for (int mult = 1; mult <= pl->max_blocks_per_sm; ++mult) {
      pl->tile_cap = cap;
      pl->grid_mult = mult;
      cudaError_t e = ragged_build_items(*pl);
      if (e != cudaSuccess) return cuda_fail(e, "ragged items");
      if (int rc = ldbp_apply_ragged(plan, taps, c, x, y, nullptr, nullptr, stream)) return rc;  // warm-up
      float tot = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        LDBP_CUDA_TRY(cudaEventRecord(e0, st));
        if (int rc = ldbp_apply_ragged(plan, taps, c, x, y, nullptr, nullptr, stream)) return rc;
        LDBP_CUDA_TRY(cudaEventRecord(e1, st));
        LDBP_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        LDBP_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        tot += ms;
      }
      if (tot < best) {
        best = tot;
        best_cap = cap;
        best_mult = mult;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pl->tile_cap = best_cap;
  pl->grid_mult = best_mult;
  cudaError_t e = ragged_build_items(*pl);
  if (e != cudaSuccess) return cuda_fail(e, "ragged items");
  if (pl->graph) {  // the captured graph refers to the old work list
    cudaGraphExecDestroy(pl->graph);
    pl->graph = nullptr;
  }
  return LDBP_OK;
}

int ldbp_ragged_set_schedule(void* plan, int32_t tile_cap, int32_t blocks_per_sm) {
  if (!plan) return fail(LDBP_EINVAL, "plan must be non-NULL");
  RaggedPlan* pl = static_cast<RaggedPlan*>(plan);
  if (tile_cap < 256 || tile_cap > kFwdS || (tile_cap & 1))
    return fail(LDBP_EINVAL, "tile_cap=%d must be even and in [256, %d]", tile_cap, kFwdS);
  if (blocks_per_sm < 1 || blocks_per_sm > pl->max_blocks_per_sm)
    return fail(LDBP_EINVAL, "blocks_per_sm=%d must be in [1, %d]", blocks_per_sm, pl->max_blocks_per_sm);
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != pl->device) return fail(LDBP_EINVAL, "plan belongs to device %d, current is %d", pl->device, dev);
  pl->tile_cap = tile_cap;
  pl->grid_mult = blocks_per_sm;
  cudaError_t e = ragged_build_items(*pl);
  if (e != cudaSuccess) return cuda_fail(e, "ragged items");
  if (pl->graph) {  // the captured graph refers to the old work list
    cudaGraphExecDestroy(pl->graph);
    pl->graph = nullptr;
  }
  return LDBP_OK;
}

int ldbp_ragged_graph_capture(void* plan, const void* taps, const float* c, const void* x, void* y) {
  if (!plan) return fail(LDBP_EINVAL, "plan must be non-NULL");
  RaggedPlan* pl = static_cast<RaggedPlan*>(plan);
  if (pl->graph) {
    cudaGraphExecDestroy(pl->graph);
    pl->graph = nullptr;
  }
  if (!pl->cap_stream) LDBP_CUDA_TRY(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
  LDBP_CUDA_TRY(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int rc = ldbp_apply_ragged(plan, taps, c, x, y, nullptr, nullptr, pl->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "graph capture");
  e = cudaGraphInstantiate(&pl->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
  return LDBP_OK;
}

int ldbp_ragged_graph_launch(void* plan, void* stream) {
  if (!plan) return fail(LDBP_EINVAL, "plan must be non-NULL");
  RaggedPlan* pl = static_cast<RaggedPlan*>(plan);
  if (!pl->graph) return fail(LDBP_EINVAL, "no graph captured for this plan");
  LDBP_CUDA_TRY(cudaGraphLaunch(pl->graph, static_cast<cudaStream_t>(stream)));
  return LDBP_OK;
}

}  // extern "C"
