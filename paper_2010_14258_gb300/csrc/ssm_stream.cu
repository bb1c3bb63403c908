// L2-resident split-step Fourier method for n = 256 x 256 samples per
// waveform (the same programs as the cluster kernel, Eqs. (6)/(8)).
//
// A waveform is viewed as a 256 x 256 matrix, sample m = m1 + 256 m2.  With
// k = k2 + 256 k1 the DFT splits into (four-step)
//   X[k2 + 256 k1] = sum_m1 W_256^{m1 k1} W_n^{m1 k2} sum_m2 x[m1 + 256 m2] W_256^{m2 k2},
// and every split-step step runs as two kernels over the batch, each reading
// and writing every sample once:
//   row kernel (per k2):  x W_n^{m1 k2} -> DFT over m1 -> spectral multiply
//                         (+ ASE) -> inverse DFT over k1 -> x W_n^{-m1 k2};
//   column kernel (per m1): inverse DFT over k2 -> Kerr rotation -> DFT over
//                         m2 of the next step (the first launch only
//                         transforms, the last one only inverts and rotates).
// The sample stays at position m1 + 256 j throughout (j = m2 in time, k2 in
// frequency); the spectral tables are stored transposed, at k1 + 256 k2.
// The batch is processed in chunks of at most 64 MB of samples (all steps of
// a chunk before the next), so that a chunk's samples and the tables stay in
// the 129 MB L2 and each launch still has 2048 blocks of work.  The kernels
// are latency-bound, not bandwidth-bound: at 256 x 65536 one 134 MB chunk and
// two 67 MB chunks time the same, 32 MB chunks 15 % slower; the row kernel runs
// 4 blocks per SM (64 registers), the column kernel 3 (its Kerr step spills
// a little below 128 registers).
//
// Each 256-point transform lives in the 16 threads of a half-warp, 16 samples
// a thread: a radix-16 DFT in registers, the twiddles W_256^{l k}, a 16 x 16
// transpose through a padded shared-memory block of the half-warp (no block
// barrier) and a second radix-16 DFT; the output is distributed like the
// input, so the inverse is the same routine on conjugated data.  All
// constants carry a tail term (radix-16 constants, W_256, W_n and the
// spectral tables), so constant rounding does not add up over many steps.
#include <cuda_fp16.h>

#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "ldbp_tile.cuh"
#include "philox.cuh"
#include "ssm.cuh"
#include "ssm_host.cuh"

namespace ldbp {

constexpr int kStNT = 256;   // threads per block = 16 half-warps
constexpr int kStPad = 17;   // float2 stride of a transpose row
constexpr long long kStChunkBytes = 64LL << 20;

struct StTables {
  const float2* w256h;   // [16 k][16 l] = W_256^{l k}, head
  const float2* w256l;   // tail
  const float2* wn;      // [k2][m1] = W_n^{m1 k2}, head
  const uint32_t* wn_lo; // tail, half2 in units of wn_scale
  float wn_scale;
};

__device__ __forceinline__ void st_load_w256(float2* sh, float2* sl, const StTables& t) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    sh[i] = t.w256h[i];
    sl[i] = t.w256l[i];
  }
}

// 256-point DFT on the 16 threads of a half-warp (lane j = 0..15 of the half):
// on entry a[i] = x[j + 16 i], on return a[k] = X[j + 16 k].  scr: the
// half-warp's [16][kStPad] region.  Contains __syncwarp (both halves of a
// warp run it together).
__device__ __forceinline__ void hw_fft256(float2 (&a)[16], int j, float2* scr, const float2* w256h,
                                          const float2* w256l) {
  dft<16>(a);
#pragma unroll
  for (int k = 1; k < 16; ++k) a[k] = cmul_hl(a[k], w256h[k * 16 + j], w256l[k * 16 + j]);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; ++k) scr[j * kStPad + k] = a[k];
  __syncwarp();
#pragma unroll
  for (int l = 0; l < 16; ++l) a[l] = scr[l * kStPad + j];
  dft<16>(a);
}

__device__ __forceinline__ void conj16(float2 (&a)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i].y = -a[i].y;
}

struct StRowParams {
  float2* y;                 // chunk base
  long long rows;            // waveforms in the chunk x 256
  StTables t;
  const float2* H;           // transposed spectral table, head
  const uint32_t* HL;        // tail
  float hl_scale;
  const float2* HN;          // transposed noise table (head) or nullptr (flat 1/n)
  float scale;
  int noise;                 // add ASE
  float noise_std, flat;
  int span, wave0;           // ASE counter word; index of the chunk's first waveform
  uint32_t counter, seed_lo, seed_hi;
};

// One row (fixed k2) per half-warp, 16 rows per block.
__global__ void __launch_bounds__(kStNT, 4) st_row_kernel(const __grid_constant__ StRowParams p) {
  __shared__ __align__(16) float2 scr_all[16 * 16 * kStPad];
  __shared__ __align__(16) float2 w256h[256], w256l[256];
  st_load_w256(w256h, w256l, p.t);
  __syncthreads();
  const int hw = threadIdx.x >> 4, j = threadIdx.x & 15;
  const long long row = (long long)blockIdx.x * 16 + hw;
  if (row >= p.rows) return;  // whole half-warps only; no block barrier follows
  const int k2 = (int)(row & 255);
  const int b = (int)(row >> 8);
  float2* scr = scr_all + hw * 16 * kStPad;
  float2* d = p.y + row * 256;
  const float2* wn = p.t.wn + k2 * 256;
  const uint32_t* wnl = p.t.wn_lo + k2 * 256;
  float2 a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int m1 = j + 16 * i;
    a[i] = cmul_hl(d[m1], __ldg(&wn[m1]), tail_h2(__ldg(&wnl[m1]), p.t.wn_scale));
  }
  hw_fft256(a, j, scr, w256h, w256l);
  // a[k] = X[k2 + 256 k1] with k1 = j + 16 k; table position k1 + 256 k2
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int k1 = j + 16 * k, pos = k1 + 256 * k2;
    float2 A = cmul_hl(a[k], __ldg(&p.H[pos]), tail_h2(__ldg(&p.HL[pos]), p.hl_scale));
    A = make_float2(A.x * p.scale, A.y * p.scale);
    if (p.noise) {
      const uint32_t kk = (uint32_t)(k2 + 256 * k1);
      const float2 g = ase_normal(kk, (uint32_t)(p.wave0 + b), (uint32_t)p.span, p.counter, p.seed_lo, p.seed_hi);
      const float2 hn = p.HN ? __ldg(&p.HN[pos]) : make_float2(p.flat, 0.f);
      A = cadd(A, cmul(hn, make_float2(g.x * p.noise_std, g.y * p.noise_std)));
    }
    a[k] = make_float2(A.x, -A.y);
  }
  hw_fft256(a, j, scr, w256h, w256l);
  conj16(a);
  // inverse twiddle W_n^{-m1 k2}
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int m1 = j + 16 * i;
    const float2 w = __ldg(&wn[m1]), wl = tail_h2(__ldg(&wnl[m1]), p.t.wn_scale);
    d[m1] = cmul_hl(a[i], make_float2(w.x, -w.y), make_float2(wl.x, -wl.y));
  }
}

// Column kernel modes.
enum StColMode : int { kStFirst = 0, kStMid = 1, kStLast = 2 };

struct StColParams {
  const float2* x;  // chunk input (read by the first launch)
  float2* y;        // chunk data
  long long cols;   // waveforms in the chunk x 16 (groups of 16 columns)
  StTables t;
  float c;          // Kerr coefficient after the inverse transform (kStMid, kStLast)
  float c_pre;      // Kerr before the first transform (kStFirst; 0: none)
};

// 16 columns (m1 in [c0, c0 + 16)) of one waveform per block, one column per
// half-warp; the 256 x 16 block of samples passes through shared memory so
// that global accesses are 128-byte rows.
template <int MODE>
__global__ void __launch_bounds__(kStNT, 3) st_col_kernel(const __grid_constant__ StColParams p) {
  __shared__ __align__(16) float2 tile[256 * kStPad];  // [j][c] during load / store, transpose scratch between
  __shared__ __align__(16) float2 w256h[256], w256l[256];
  st_load_w256(w256h, w256l, p.t);
  const int t = threadIdx.x, hw = t >> 4, j = t & 15;
  const long long g = blockIdx.x;
  if (g >= p.cols) return;  // uniform per block
  const long long b = g >> 4;
  const int c0 = (int)(g & 15) * 16;
  const float2* src = (MODE == kStFirst ? p.x : p.y) + b * 65536 + c0;
  float2* dst = p.y + b * 65536 + c0;
  // coalesced load: thread t reads column t % 16 of rows t / 16 + 16 r
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int row = hw + 16 * r;
    float2 v = src[row * 256 + j];
    if (MODE == kStFirst && p.c_pre != 0.f) v = kerr_rotate_precise<true>(v, p.c_pre);
    tile[row * kStPad + j] = v;
  }
  __syncthreads();
  // half-warp hw owns column hw: a[i] = sample of row j + 16 i
  float2 a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = tile[(j + 16 * i) * kStPad + hw];
  __syncthreads();  // the tile becomes transpose scratch
  float2* scr = tile + hw * 16 * kStPad;
  if (MODE != kStFirst) {
    // inverse over k2: conj o DFT o conj (1 / n is in the spectral table)
    conj16(a);
    hw_fft256(a, j, scr, w256h, w256l);
    conj16(a);
    if (p.c != 0.f) tile_kerr<16>(a, p.c);
  }
  if (MODE != kStLast) hw_fft256(a, j, scr, w256h, w256l);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[(j + 16 * i) * kStPad + hw] = a[i];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int row = hw + 16 * r;
    dst[row * 256 + j] = tile[row * kStPad + j];
  }
}

// Transposed copy of a spectral table: out[k1 + 256 k2] = in[k2 + 256 k1].
__global__ void st_transpose_kernel(const float2* __restrict__ in, const uint32_t* __restrict__ in_lo,
                                    float2* __restrict__ out, uint32_t* __restrict__ out_lo) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= 65536) return;
  const int k1 = pos & 255, k2 = pos >> 8;
  out[pos] = in[k2 + 256 * k1];
  if (in_lo) out_lo[pos] = in_lo[k2 + 256 * k1];
}

// ------------------------------------------------------------------ host
static const double kPiSt = 3.14159265358979323846;

// Head/tail float pairs of exp(-j 2 pi e / N) (head = float rounding, tail =
// float rounding of the remainder).
static void hl_pair(double ang, float2* h, float2* l) {
  const double c = std::cos(ang), s = std::sin(ang);
  *h = make_float2((float)c, (float)s);
  *l = make_float2((float)(c - (double)h->x), (float)(s - (double)h->y));
}

struct StCache {
  float2 *w256h = nullptr, *w256l = nullptr, *wn = nullptr;
  uint32_t* wn_lo = nullptr;
  float wn_scale = 1.f;
};
static std::mutex g_st_mu;
static std::map<int, StCache> g_st_cache;  // per device

static int st_tables(StTables* t) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_st_mu);
  StCache& c = g_st_cache[dev];
  if (!c.wn) {
    std::vector<float2> h256(256), l256(256);
    for (int k = 0; k < 16; ++k)
      for (int l = 0; l < 16; ++l) hl_pair(-2.0 * kPiSt * (double)((l * k) % 256) / 256.0, &h256[k * 16 + l], &l256[k * 16 + l]);
    std::vector<float2> wh(65536);
    std::vector<double> rem(2 * 65536);
    double m = 0.0;
    for (int k2 = 0; k2 < 256; ++k2)
      for (int m1 = 0; m1 < 256; ++m1) {
        float2 h, l;
        hl_pair(-2.0 * kPiSt * (double)((m1 * k2) % 65536) / 65536.0, &h, &l);
        const int pos = k2 * 256 + m1;
        wh[pos] = h;
        rem[2 * pos] = l.x;
        rem[2 * pos + 1] = l.y;
        m = std::max(m, std::max(std::fabs(rem[2 * pos]), std::fabs(rem[2 * pos + 1])));
      }
    c.wn_scale = m > 0.0 ? (float)m : 1.f;
    std::vector<uint32_t> wl(65536);
    for (int i = 0; i < 65536; ++i) {
      const __half2 q = __floats2half2_rn((float)(rem[2 * i] / c.wn_scale), (float)(rem[2 * i + 1] / c.wn_scale));
      memcpy(&wl[i], &q, sizeof(uint32_t));
    }
    cudaError_t e = cudaMalloc(&c.w256h, 256 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&c.w256l, 256 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&c.wn, 65536 * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&c.wn_lo, 65536 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(c.w256h, h256.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.w256l, l256.data(), 256 * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.wn, wh.data(), 65536 * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c.wn_lo, wl.data(), 65536 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      c = StCache{};
      return cuda_fail(e, "split-step (L2-resident) twiddle tables");
    }
  }
  *t = StTables{c.w256h, c.w256l, c.wn, c.wn_lo, c.wn_scale};
  return 0;
}

// Transposed copies of the program's tables (made once per program).
static int st_program_tables(const DeviceProgram& dp_in, cudaStream_t st) {
  DeviceProgram& dp = const_cast<DeviceProgram&>(dp_in);
  std::lock_guard<std::mutex> lk(g_st_mu);
  if (dp.st_tabs.size() == dp.tabs.size()) return 0;
  for (size_t i = dp.st_tabs.size(); i < dp.tabs.size(); ++i) {
    float2* h = nullptr;
    uint32_t* l = nullptr;
    LDBP_CUDA_TRY(cudaMalloc(&h, 65536 * sizeof(float2)));
    LDBP_CUDA_TRY(cudaMalloc(&l, 65536 * sizeof(uint32_t)));
    st_transpose_kernel<<<256, 256, 0, st>>>(dp.tabs[i], dp.tabs_lo[i], h, l);
    LDBP_CUDA_TRY(cudaGetLastError());
    LDBP_CUDA_TRY(cudaStreamSynchronize(st));
    dp.st_tabs.push_back(h);
    dp.st_tabs_lo.push_back(l);
  }
  return 0;
}

bool ssm_stream_supported(long long n) { return n == 65536; }

int run_program_stream(const DeviceProgram& dp, const void* x, void* y, long long n, int batch, uint64_t seed,
                       uint64_t counter, cudaStream_t st) {
  if (!ssm_stream_supported(n)) return fail(LDBP_EINVAL, "L2-resident split step needs n = 65536");
  StTables t;
  if (int rc = st_tables(&t)) return rc;
  if (int rc = st_program_tables(dp, st)) return rc;
  const long long wave_bytes = n * (long long)sizeof(float2);
  const int chunk = (int)std::max(1LL, std::min((long long)batch, kStChunkBytes / wave_bytes));
  const float2* X = static_cast<const float2*>(x);
  float2* Y = static_cast<float2*>(y);
  for (int w0 = 0; w0 < batch; w0 += chunk) {
    const int nw = std::min(chunk, batch - w0);
    StColParams cp;
    cp.x = X + (long long)w0 * n;
    cp.y = Y + (long long)w0 * n;
    cp.cols = (long long)nw * 16;
    cp.t = t;
    cp.c = 0.f;
    cp.c_pre = dp.c_pre;
    const unsigned col_grid = (unsigned)cp.cols;
    st_col_kernel<kStFirst><<<col_grid, kStNT, 0, st>>>(cp);
    StRowParams rp;
    rp.y = Y + (long long)w0 * n;
    rp.rows = (long long)nw * 256;
    rp.t = t;
    rp.flat = 1.0f / (float)n;
    rp.noise_std = dp.noise_std;
    rp.wave0 = w0;
    rp.counter = (uint32_t)(counter & 0xffffffffu);
    rp.seed_lo = (uint32_t)(seed & 0xffffffffu);
    rp.seed_hi = (uint32_t)(seed >> 32);
    const unsigned row_grid = (unsigned)((rp.rows + 15) / 16);
    for (int s = 0; s < dp.nsteps; ++s) {
      const SsmStep& ss = dp.host_steps[(size_t)s];
      rp.H = dp.st_tabs[(size_t)ss.tab];
      rp.HL = dp.st_tabs_lo[(size_t)ss.tab];
      rp.hl_scale = dp.tabs_lo_scale[(size_t)ss.tab];
      rp.HN = ss.noise_tab >= 0 ? dp.st_tabs[(size_t)ss.noise_tab] : nullptr;
      rp.noise = ss.noise_tab > -2;
      rp.scale = ss.scale;
      rp.span = ss.span;
      st_row_kernel<<<row_grid, kStNT, 0, st>>>(rp);
      cp.c = ss.c;
      if (s + 1 < dp.nsteps)
        st_col_kernel<kStMid><<<col_grid, kStNT, 0, st>>>(cp);
      else
        st_col_kernel<kStLast><<<col_grid, kStNT, 0, st>>>(cp);
    }
  }
  LDBP_CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // namespace ldbp
