// L2-resident split-step Fourier method for n = N1 x 256 samples per
// waveform, N1 = 256 or 512 (the same programs as the cluster kernel,
// Eqs. (6)/(8)).  At n = 32768 (N1 = 128) the cluster kernel is faster
// (9.6 against 10.9 ps per sample-step at 512 waveforms), so that length
// stays there.
//
// A waveform is viewed as an N1 x 256 matrix, sample m = m1 + N1 m2.  With
// k = k2 + 256 k1 the DFT splits into (four-step)
//   X[k2 + 256 k1] = sum_m1 W_N1^{m1 k1} W_n^{m1 k2} sum_m2 x[m1 + N1 m2] W_256^{m2 k2},
// and every split-step step runs as two kernels over the batch, each reading
// and writing every sample once:
//   row kernel (per k2):  x W_n^{m1 k2} -> DFT over m1 -> spectral multiply
//                         (+ ASE) -> inverse DFT over k1 -> x W_n^{-m1 k2};
//   column kernel (per m1): inverse DFT over k2 -> Kerr rotation -> DFT over
//                         m2 of the next step (the first launch only
//                         transforms, the last one only inverts and rotates).
// The sample stays at position m1 + N1 j throughout (j = m2 in time, k2 in
// frequency); the spectral tables are stored transposed, at k1 + N1 k2.
// The batch is processed in chunks of at most 64 MB of samples (all steps of
// a chunk before the next), so that a chunk's samples and the tables stay in
// the 129 MB L2 and each launch still has thousands of blocks.  The kernels
// are latency-bound, not bandwidth-bound: at 256 x 65536 one 134 MB chunk and
// two 67 MB chunks time the same, 32 MB chunks 15 % slower; the row kernel runs
// 4 blocks per SM, the column kernel 3 (its Kerr step spills a little below
// 128 registers).
//
// A transform of N = TPR x E points lives in TPR consecutive threads, E
// samples a thread (thread t holds x[t + TPR i]): a radix-E DFT in registers,
// the twiddles W_N^{t k}, a TPR x E transpose through a padded shared-memory
// block of that thread group (no block barrier) and radix-TPR DFTs; the
// output is distributed like the input (thread t holds X[t + TPR q]), so the
// inverse is the same routine on conjugated data.  Column transforms and
// rows of 256: 16 x 16 on a half-warp.  Rows of 512: 16 x 32 on a warp, the
// radix-32 stage split over the two half-warps (a radix-2 butterfly through
// lane shuffles), with the transposed algorithm as the inverse.  All
// constants carry a tail term (radix constants, W_N, W_n and the spectral
// tables), so constant rounding does not add up over many steps.
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

constexpr int kStNT = 256;      // threads per column-kernel block
constexpr int kStCol = 256;     // column transform length (the m2 / k2 axis)
constexpr long long kStChunkBytes = 64LL << 20;

// Geometry of an N-point transform on TPR threads with E samples each, and
// the threads per block of the row kernel for that length (its per-group
// transpose scratch stays within 48 KB of static shared memory).
template <int N>
struct StGeo;
template <>
struct StGeo<256> {
  static constexpr int TPR = 16, E = 16, NT = 256;
};
template <>
struct StGeo<512> {
  static constexpr int TPR = 32, E = 16, NT = 256;
};

// Twiddle tables of one N1: W_N1 for the row transforms, W_256 for the
// column transforms ([k][t] = W_N^{t k}, head and tail), and W_n at [k2][m1].
struct StTables {
  const float2 *wrh, *wrl;   // [E][TPR] row-transform twiddles (N1 points)
  const float2 *wch, *wcl;   // [16][16] column-transform twiddles (256 points)
  const float2* wn;          // [256][N1] = W_n^{m1 k2}, head
  const uint32_t* wn_lo;     // tail, half2 in units of wn_scale
  float wn_scale;
};

// N-point DFT on the TPR threads of a group (t = 0..TPR-1): on entry
// a[i] = x[t + TPR i], on return a[q] = X[t + TPR q].  scr: the group's
// [TPR][E + 1] region; tw*: [E][TPR] twiddles W_N^{t k}.  With k = k1 + E k2
// (k1 < E, k2 < TPR): a radix-E DFT over i, the twiddle W_N^{t k1}, the
// transpose, and a radix-TPR DFT over t for each k1 = t' + TPR b this thread
// owns.  Contains __syncwarp (every group of the warp runs it together).
template <int N>
__device__ __forceinline__ void st_fft(float2 (&a)[StGeo<N>::E], int t, float2* scr, const float2* twh,
                                       const float2* twl) {
  constexpr int TPR = StGeo<N>::TPR, E = StGeo<N>::E, S = E + 1, NB = E / TPR;
  static_assert(E >= TPR, "one radix-TPR pass per owned output column");
  dft<E>(a);
#pragma unroll
  for (int k = 1; k < E; ++k) a[k] = cmul_hl(a[k], twh[k * TPR + t], twl[k * TPR + t]);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < E; ++k) scr[t * S + k] = a[k];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    float2 c[TPR];
#pragma unroll
    for (int l = 0; l < TPR; ++l) c[l] = scr[l * S + t + TPR * b];
    dft<TPR>(c);
    // c[k2] = X[t + TPR b + E k2] = X[t + TPR (b + NB k2)]
#pragma unroll
    for (int k = 0; k < TPR; ++k) a[b + NB * k] = c[k];
  }
}

template <int E>
__device__ __forceinline__ void st_conj(float2 (&a)[E]) {
#pragma unroll
  for (int i = 0; i < E; ++i) a[i].y = -a[i].y;
}

// 512-point transform on the 32 lanes of a warp, 16 samples a lane.
// Forward (input a[i] = x[t + 32 i]): with k = k1 + 16 k2 (k1 < 16, k2 < 32),
// a radix-16 DFT over i, the twiddle W_512^{t k1} and a 32 x 16 transpose;
// lane t then owns column k1 = t % 16 and the half p = t / 16 of its 32-point
// DFT over t: a radix-16 DFT of the samples 2 m + p (m < 16), W_32^k on the
// odd half, and the radix-2 butterfly with the partner lane t ^ 16.  Output:
// a[k] = X[(t % 16) + 16 k + 256 (t / 16)].
// Inverse direction (st_fft512_t): the transposed algorithm, the same stages
// in reverse order (the DFT matrix is symmetric), which consumes that output
// distribution and returns a[i] = x[t + 32 i]; conj o st_fft512_t o conj is
// then the exact algebraic inverse of st_fft512 up to the factor 512.
// scr: the warp's [32][17] region; tw*: [16][32] twiddles W_512^{t k1}.
__device__ __forceinline__ void st_butterfly_x16(float2 (&a)[16], int p) {
  // (u, w) -> (u + w, u - w) across lanes t and t ^ 16: lane p = 0 holds u,
  // p = 1 holds w; u - w is formed as u + (-w) (the negation is exact)
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float2 v = make_float2(__shfl_xor_sync(0xffffffffu, a[k].x, 16), __shfl_xor_sync(0xffffffffu, a[k].y, 16));
    const float2 own = p ? make_float2(-a[k].x, -a[k].y) : a[k];
    a[k] = padd(own, v);
  }
}

__device__ __forceinline__ void st_tw32_odd(float2 (&a)[16], int p) {
  if (p) tw32_loop<1>(a);
}

__device__ __forceinline__ void st_fft512(float2 (&a)[16], int t, float2* scr, const float2* twh,
                                          const float2* twl) {
  constexpr int S = 17;
  const int k1 = t & 15, p = t >> 4;
  dft<16>(a);
#pragma unroll
  for (int k = 1; k < 16; ++k) a[k] = cmul_hl(a[k], twh[k * 32 + t], twl[k * 32 + t]);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; ++k) scr[t * S + k] = a[k];
  __syncwarp();
#pragma unroll
  for (int m = 0; m < 16; ++m) a[m] = scr[(2 * m + p) * S + k1];
  dft<16>(a);
  st_tw32_odd(a, p);
  st_butterfly_x16(a, p);
}

__device__ __forceinline__ void st_fft512_t(float2 (&a)[16], int t, float2* scr, const float2* twh,
                                            const float2* twl) {
  constexpr int S = 17;
  const int k1 = t & 15, p = t >> 4;
  st_butterfly_x16(a, p);
  st_tw32_odd(a, p);
  dft<16>(a);
  __syncwarp();
#pragma unroll
  for (int m = 0; m < 16; ++m) scr[(2 * m + p) * S + k1] = a[m];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = scr[t * S + k];
#pragma unroll
  for (int k = 1; k < 16; ++k) a[k] = cmul_hl(a[k], twh[k * 32 + t], twl[k * 32 + t]);
  dft<16>(a);
}

// Row-frequency index held in a[q] by lane t of a row group after the forward
// row transform.
template <int N1>
__device__ __forceinline__ int st_krow(int t, int q) {
  if constexpr (N1 == 512)
    return (t & 15) + 16 * q + 256 * (t >> 4);
  else
    return t + StGeo<N1>::TPR * q;
}

template <int N1>
__device__ __forceinline__ void st_row_fwd(float2 (&a)[StGeo<N1>::E], int t, float2* scr, const float2* twh,
                                           const float2* twl) {
  if constexpr (N1 == 512)
    st_fft512(a, t, scr, twh, twl);
  else
    st_fft<N1>(a, t, scr, twh, twl);
}

// Inverse row transform (without the conjugations around it).
template <int N1>
__device__ __forceinline__ void st_row_inv(float2 (&a)[StGeo<N1>::E], int t, float2* scr, const float2* twh,
                                           const float2* twl) {
  if constexpr (N1 == 512)
    st_fft512_t(a, t, scr, twh, twl);
  else
    st_fft<N1>(a, t, scr, twh, twl);
}

__device__ __forceinline__ void st_load_tw(float2* dh, float2* dl, const float2* sh, const float2* sl, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    dh[i] = sh[i];
    dl[i] = sl[i];
  }
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

// One row (fixed k2) per group of TPR threads, NT / TPR rows per block.
template <int N1>
__global__ void __launch_bounds__(StGeo<N1>::NT, 4) st_row_kernel(const __grid_constant__ StRowParams p) {
  constexpr int TPR = StGeo<N1>::TPR, E = StGeo<N1>::E, G = StGeo<N1>::NT / TPR;
  __shared__ __align__(16) float2 scr_all[G * TPR * (E + 1)];
  __shared__ __align__(16) float2 twh[N1], twl[N1];
  st_load_tw(twh, twl, p.t.wrh, p.t.wrl, N1);
  __syncthreads();
  const int g = threadIdx.x / TPR, t = threadIdx.x % TPR;
  const long long row = (long long)blockIdx.x * G + g;
  if (row >= p.rows) return;  // whole blocks only (rows is a multiple of 256 and of G); no block barrier follows
  const int k2 = (int)(row & 255);
  const int b = (int)(row >> 8);
  float2* scr = scr_all + g * TPR * (E + 1);
  float2* d = p.y + row * N1;
  const float2* wn = p.t.wn + k2 * N1;
  const uint32_t* wnl = p.t.wn_lo + k2 * N1;
  float2 a[E];
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int m1 = t + TPR * i;
    a[i] = cmul_hl(d[m1], __ldg(&wn[m1]), tail_h2(__ldg(&wnl[m1]), p.t.wn_scale));
  }
  st_row_fwd<N1>(a, t, scr, twh, twl);
  // a[q] = X[k2 + 256 k1] with k1 = st_krow(t, q); table position k1 + N1 k2
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int k1 = st_krow<N1>(t, q), pos = k1 + N1 * k2;
    float2 A = cmul_hl(a[q], __ldg(&p.H[pos]), tail_h2(__ldg(&p.HL[pos]), p.hl_scale));
    A = make_float2(A.x * p.scale, A.y * p.scale);
    if (p.noise) {
      const uint32_t kk = (uint32_t)(k2 + 256 * k1);
      const float2 gn = ase_normal(kk, (uint32_t)(p.wave0 + b), (uint32_t)p.span, p.counter, p.seed_lo, p.seed_hi);
      const float2 hn = p.HN ? __ldg(&p.HN[pos]) : make_float2(p.flat, 0.f);
      A = cadd(A, cmul(hn, make_float2(gn.x * p.noise_std, gn.y * p.noise_std)));
    }
    a[q] = make_float2(A.x, -A.y);
  }
  st_row_inv<N1>(a, t, scr, twh, twl);
  st_conj<E>(a);
  // inverse twiddle W_n^{-m1 k2}
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const int m1 = t + TPR * i;
    const float2 w = __ldg(&wn[m1]), wl = tail_h2(__ldg(&wnl[m1]), p.t.wn_scale);
    d[m1] = cmul_hl(a[i], make_float2(w.x, -w.y), make_float2(wl.x, -wl.y));
  }
}

// Column kernel modes.
enum StColMode : int { kStFirst = 0, kStMid = 1, kStLast = 2 };

struct StColParams {
  const float2* x;  // chunk input (read by the first launch)
  float2* y;        // chunk data
  long long cols;   // waveforms in the chunk x N1 / 16 (groups of 16 columns)
  StTables t;
  float c;          // Kerr coefficient after the inverse transform (kStMid, kStLast)
  float c_pre;      // Kerr before the first transform (kStFirst; 0: none)
};

// 16 columns (m1 in [c0, c0 + 16)) of one waveform per block, one column per
// half-warp; the 256 x 16 block of samples passes through shared memory so
// that global accesses are 128-byte rows.
template <int N1, int MODE>
__global__ void __launch_bounds__(kStNT, 3) st_col_kernel(const __grid_constant__ StColParams p) {
  constexpr int S = 17;                                   // float2 stride of a tile row
  __shared__ __align__(16) float2 tile[kStCol * S];      // [j][c] during load / store, transpose scratch between
  __shared__ __align__(16) float2 twh[256], twl[256];
  st_load_tw(twh, twl, p.t.wch, p.t.wcl, 256);
  const int tid = threadIdx.x, hw = tid >> 4, j = tid & 15;
  const long long g = blockIdx.x;
  if (g >= p.cols) return;  // uniform per block
  constexpr int GPW = N1 / 16;  // column groups per waveform
  const long long b = g / GPW;
  const int c0 = (int)(g % GPW) * 16;
  constexpr long long n = (long long)N1 * kStCol;
  const float2* src = (MODE == kStFirst ? p.x : p.y) + b * n + c0;
  float2* dst = p.y + b * n + c0;
  // coalesced load: thread tid reads column tid % 16 of rows tid / 16 + 16 r
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int row = hw + 16 * r;
    float2 v = src[(long long)row * N1 + j];
    if (MODE == kStFirst && p.c_pre != 0.f) v = kerr_rotate_precise<true>(v, p.c_pre);
    tile[row * S + j] = v;
  }
  __syncthreads();
  // half-warp hw owns column hw: a[i] = sample of row j + 16 i
  float2 a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = tile[(j + 16 * i) * S + hw];
  __syncthreads();  // the tile becomes transpose scratch
  float2* scr = tile + hw * 16 * S;
  if (MODE != kStFirst) {
    // inverse over k2: conj o DFT o conj (1 / n is in the spectral table)
    st_conj<16>(a);
    st_fft<256>(a, j, scr, twh, twl);
    st_conj<16>(a);
    if (p.c != 0.f) tile_kerr<16>(a, p.c);
  }
  if (MODE != kStLast) st_fft<256>(a, j, scr, twh, twl);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 16; ++i) tile[(j + 16 * i) * S + hw] = a[i];
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int row = hw + 16 * r;
    dst[(long long)row * N1 + j] = tile[row * S + j];
  }
}

// Transposed copy of a spectral table: out[k1 + N1 k2] = in[k2 + 256 k1].
__global__ void st_transpose_kernel(const float2* __restrict__ in, const uint32_t* __restrict__ in_lo,
                                    float2* __restrict__ out, uint32_t* __restrict__ out_lo, int n1) {
  const int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= n1 * kStCol) return;
  const int k1 = pos % n1, k2 = pos / n1;
  out[pos] = in[k2 + kStCol * k1];
  if (in_lo) out_lo[pos] = in_lo[k2 + kStCol * k1];
}

// ------------------------------------------------------------------ host
static const double kPiSt = 3.14159265358979323846;

// Head/tail float pairs of exp(-j ang) (head = float rounding, tail = float
// rounding of the remainder).
static void hl_pair(double ang, float2* h, float2* l) {
  const double c = std::cos(ang), s = -std::sin(ang);
  *h = make_float2((float)c, (float)s);
  *l = make_float2((float)(c - (double)h->x), (float)(s - (double)h->y));
}

// [k][t] = W_N^{t k} = exp(-j 2 pi t k / N) for an N = TPR x E transform.
static void transform_twiddles(int N, int TPR, int E, std::vector<float2>* h, std::vector<float2>* l) {
  h->assign((size_t)N, make_float2(0.f, 0.f));
  l->assign((size_t)N, make_float2(0.f, 0.f));
  for (int k = 0; k < E; ++k)
    for (int t = 0; t < TPR; ++t)
      hl_pair(2.0 * kPiSt * (double)((t * k) % N) / (double)N, &(*h)[(size_t)(k * TPR + t)],
              &(*l)[(size_t)(k * TPR + t)]);
}

struct StCache {
  float2 *wrh = nullptr, *wrl = nullptr, *wch = nullptr, *wcl = nullptr, *wn = nullptr;
  uint32_t* wn_lo = nullptr;
  float wn_scale = 1.f;
};
static std::mutex g_st_mu;
static std::map<std::pair<int, int>, StCache> g_st_cache;  // (device, N1)

template <typename T>
static cudaError_t st_upload(const std::vector<T>& h, T** out) {
  cudaError_t e = cudaMalloc(out, h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*out, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static int st_tables(int n1, int tpr, int e, StTables* t) {
  int dev = 0;
  LDBP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_st_mu);
  StCache& c = g_st_cache[{dev, n1}];
  if (!c.wn) {
    std::vector<float2> rh, rl, ch, cl;
    transform_twiddles(n1, tpr, e, &rh, &rl);
    transform_twiddles(kStCol, 16, 16, &ch, &cl);
    const long long n = (long long)n1 * kStCol;
    std::vector<float2> wh((size_t)n);
    std::vector<double> rem(2 * (size_t)n);
    double m = 0.0;
    for (int k2 = 0; k2 < kStCol; ++k2)
      for (int m1 = 0; m1 < n1; ++m1) {
        float2 h, l;
        hl_pair(2.0 * kPiSt * (double)(((long long)m1 * k2) % n) / (double)n, &h, &l);
        const size_t pos = (size_t)k2 * n1 + m1;
        wh[pos] = h;
        rem[2 * pos] = l.x;
        rem[2 * pos + 1] = l.y;
        m = std::max(m, std::max(std::fabs(rem[2 * pos]), std::fabs(rem[2 * pos + 1])));
      }
    c.wn_scale = m > 0.0 ? (float)m : 1.f;
    std::vector<uint32_t> wl((size_t)n);
    for (size_t i = 0; i < (size_t)n; ++i) {
      const __half2 q = __floats2half2_rn((float)(rem[2 * i] / c.wn_scale), (float)(rem[2 * i + 1] / c.wn_scale));
      memcpy(&wl[i], &q, sizeof(uint32_t));
    }
    cudaError_t er = st_upload(rh, &c.wrh);
    if (er == cudaSuccess) er = st_upload(rl, &c.wrl);
    if (er == cudaSuccess) er = st_upload(ch, &c.wch);
    if (er == cudaSuccess) er = st_upload(cl, &c.wcl);
    if (er == cudaSuccess) er = st_upload(wh, &c.wn);
    if (er == cudaSuccess) er = st_upload(wl, &c.wn_lo);
    if (er != cudaSuccess) {
      c = StCache{};
      return cuda_fail(er, "split-step (L2-resident) twiddle tables");
    }
  }
  *t = StTables{c.wrh, c.wrl, c.wch, c.wcl, c.wn, c.wn_lo, c.wn_scale};
  return 0;
}

// Transposed copies of the program's tables (made once per program).
static int st_program_tables(const DeviceProgram& dp_in, int n1, cudaStream_t st) {
  DeviceProgram& dp = const_cast<DeviceProgram&>(dp_in);
  std::lock_guard<std::mutex> lk(g_st_mu);
  if (dp.st_tabs.size() == dp.tabs.size()) return 0;
  const int n = n1 * kStCol;
  for (size_t i = dp.st_tabs.size(); i < dp.tabs.size(); ++i) {
    float2* h = nullptr;
    uint32_t* l = nullptr;
    LDBP_CUDA_TRY(cudaMalloc(&h, (size_t)n * sizeof(float2)));
    LDBP_CUDA_TRY(cudaMalloc(&l, (size_t)n * sizeof(uint32_t)));
    st_transpose_kernel<<<(n + 255) / 256, 256, 0, st>>>(dp.tabs[i], dp.tabs_lo[i], h, l, n1);
    LDBP_CUDA_TRY(cudaGetLastError());
    LDBP_CUDA_TRY(cudaStreamSynchronize(st));
    dp.st_tabs.push_back(h);
    dp.st_tabs_lo.push_back(l);
  }
  return 0;
}

// Whether a batch runs here rather than on the cluster kernel (measured, at
// 25 x 80 km, 1 and 4 StPS): n = 65536 from 24 waveforms (at 8 the cluster
// kernel takes 1.40 ms against 1.82, at 24 both 2.8 ms, at 256 13.5 against
// 9.9 ps per sample-step), n = 131072 from 8 (3.57 against 3.09 ms at 8, 19.0
// against 12.6 ps at 128).  Below 8 waveforms of 131072 samples the cluster
// kernel finishes in one wave of 16-block clusters.
bool ssm_stream_preferred(long long n, int batch) {
  if (n == 256LL * kStCol) return batch >= 24;
  if (n == 512LL * kStCol) return batch >= 8;
  return false;
}

template <int N1>
static int run_stream(const DeviceProgram& dp, const void* x, void* y, int batch, uint64_t seed, uint64_t counter,
                      cudaStream_t st) {
  constexpr int TPR = StGeo<N1>::TPR, E = StGeo<N1>::E, G = StGeo<N1>::NT / TPR;
  constexpr long long n = (long long)N1 * kStCol;
  StTables t;
  if (int rc = st_tables(N1, TPR, E, &t)) return rc;
  if (int rc = st_program_tables(dp, N1, st)) return rc;
  const int chunk = (int)std::max(1LL, std::min((long long)batch, kStChunkBytes / (n * (long long)sizeof(float2))));
  const float2* X = static_cast<const float2*>(x);
  float2* Y = static_cast<float2*>(y);
  for (int w0 = 0; w0 < batch; w0 += chunk) {
    const int nw = std::min(chunk, batch - w0);
    StColParams cp;
    cp.x = X + (long long)w0 * n;
    cp.y = Y + (long long)w0 * n;
    cp.cols = (long long)nw * (N1 / 16);
    cp.t = t;
    cp.c = 0.f;
    cp.c_pre = dp.c_pre;
    const unsigned col_grid = (unsigned)cp.cols;
    st_col_kernel<N1, kStFirst><<<col_grid, kStNT, 0, st>>>(cp);
    StRowParams rp;
    rp.y = Y + (long long)w0 * n;
    rp.rows = (long long)nw * kStCol;
    rp.t = t;
    rp.flat = 1.0f / (float)n;
    rp.noise_std = dp.noise_std;
    rp.wave0 = w0;
    rp.counter = (uint32_t)(counter & 0xffffffffu);
    rp.seed_lo = (uint32_t)(seed & 0xffffffffu);
    rp.seed_hi = (uint32_t)(seed >> 32);
    const unsigned row_grid = (unsigned)((rp.rows + G - 1) / G);
    for (int s = 0; s < dp.nsteps; ++s) {
      const SsmStep& ss = dp.host_steps[(size_t)s];
      rp.H = dp.st_tabs[(size_t)ss.tab];
      rp.HL = dp.st_tabs_lo[(size_t)ss.tab];
      rp.hl_scale = dp.tabs_lo_scale[(size_t)ss.tab];
      rp.HN = ss.noise_tab >= 0 ? dp.st_tabs[(size_t)ss.noise_tab] : nullptr;
      rp.noise = ss.noise_tab > -2;
      rp.scale = ss.scale;
      rp.span = ss.span;
      st_row_kernel<N1><<<row_grid, StGeo<N1>::NT, 0, st>>>(rp);
      cp.c = ss.c;
      if (s + 1 < dp.nsteps)
        st_col_kernel<N1, kStMid><<<col_grid, kStNT, 0, st>>>(cp);
      else
        st_col_kernel<N1, kStLast><<<col_grid, kStNT, 0, st>>>(cp);
    }
  }
  LDBP_CUDA_TRY(cudaGetLastError());
  return 0;
}

int run_program_stream(const DeviceProgram& dp, const void* x, void* y, long long n, int batch, uint64_t seed,
                       uint64_t counter, cudaStream_t st) {
  switch (n / kStCol) {
    case 256: return run_stream<256>(dp, x, y, batch, seed, counter, st);
    case 512: return run_stream<512>(dp, x, y, batch, seed, counter, st);
    default: return fail(LDBP_EINVAL, "L2-resident split step needs n = 256 x 256 or 512 x 256");
  }
}

}  // namespace ldbp
