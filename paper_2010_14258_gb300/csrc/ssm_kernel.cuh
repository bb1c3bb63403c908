// Cluster-resident split-step Fourier kernel (plain SSM channel and full DBP).
//
// Every step of Eqs. (6)/(8) is  u <- sigma( iDFT( H . DFT(u) ) )  (with the
// half-steps of the symmetric method merged across step boundaries, and the
// ASE of an amplifier added in the spectral domain).  A waveform of
// n = P * N2 samples (N2 a power of two, P in 1, 2, 4, 8, 16 or, for the
// 3 * 2^k grids of 6 samples/symbol, 3, 6, 12) lives in the shared memory of
// a thread-block cluster of P blocks for ALL steps: HBM is touched once to
// load and once to store.
//
// Transform (Cooley-Tukey with n = P * N2, "four-step" split):
//   block r holds the decimated sequence x_r[m2] = x[r + P m2];
//   1. local N2-point Stockham FFT in shared memory (radix 16, conflict-free
//      padded layout): Y_r[k2];
//   2. every block pushes chunk q of Y_r (a range of k2) into block q's receive
//      buffer by remote (DSMEM) stores; block q then, for each of its k2,
//      multiplies Y_r[k2] by exp(-j 2 pi r k2 / n), runs the P-point DFT over
//      r -> X[k2 + N2 k1], applies the step's spectral multiply (and noise),
//      conjugates, runs the P-point DFT again, multiplies by the same twiddles
//      and pushes the value for r back to block r;
//   3. local N2-point transform of the conjugated data with the passes of
//      step 1 transposed and in reverse order (decimation in frequency);
//      conjugating its output gives the inverse transform, and the Kerr
//      rotation is applied in registers before the result is stored.
//
// Accuracy over thousands of steps.  The inverse is the exact algebraic
// inverse of the forward transform built from the same rounded constants:
// every pass of step 3 is the transpose of a pass of step 1, the twiddle
// tables hold float pairs with |w|^2 = 1 to about 1e-9 (chosen on the host),
// and the radix-8/16 constants carry a tail term.  Then a constant's angle
// error cancels between the two transforms instead of adding up step after
// step, and no constant scales a sample path by |w| != 1.  The spectral
// tables hold a head and a tail float per value for the same reason: the
// same table multiplies the spectrum at every step.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"
#include "fft.cuh"
#include "ssm.cuh"
#include "philox.cuh"
#include "ldbp_tile.cuh"

namespace cg = cooperative_groups;

namespace ldbp {

constexpr int kSsmE = 16;  // complex elements per thread

// Twiddle layout (one device buffer per (n, P, N2)):
//   [(q-1) N2 + k2]           = exp(-j 2 pi q k2 / n),     q = 1..P-1 (cluster step)
//   stage(Ns) + [(q-1) Ns + k] = exp(-j 2 pi q k / (Ns R)), q = 1..R-1 (local pass with Ns > 1)
// so that consecutive threads read consecutive entries.
__host__ __device__ constexpr int ssm_stage_offset(int logn2, int logns_target) {
  int off = 0, logns = 0;
  while (logns < logns_target) {
    const int logr = (logns == 0 && (logn2 % 4) != 0) ? (logn2 % 4) : 4;
    if (logns > 0) off += ((1 << logr) - 1) << logns;
    logns += logr;
  }
  return off;
}

// One radix-R Stockham pass of the local N2-point forward FFT (decimation in
// time; in place, loads complete before stores).  Ns = product of the
// earlier radices.
// PUSH_P > 1 (last pass of the forward transform in a P-block cluster): the
// outputs go straight to their owners' receive buffers (st.async counted on
// the owner's bars[0]) instead of local shared memory: output k2 belongs to
// block k2 / C at position r C + k2 % C, C = ceil(N2 / P).
struct SsmPush {
  uint32_t recv_l, bar0_l;
  int r;
};

// t: the thread's index among the N2 / 16 threads working on sbuf; threads
// with active == false (other work in the same block) only take part in the
// barriers.
template <int LOGN2, int LOGNS, int LOGR, int PUSH_P = 0>
__device__ __forceinline__ void ssm_pass(float2* sbuf, const float2* __restrict__ stw, int t, bool active,
                                         const SsmPush& push = SsmPush{0u, 0u, 0}) {
  constexpr int N2 = 1 << LOGN2, R = 1 << LOGR, Ns = 1 << LOGNS, NT = N2 / kSsmE, NB = kSsmE / R;
  const float2* __restrict__ tw = stw + ssm_stage_offset(LOGN2, LOGNS);
  float2 a[kSsmE];
  if (active) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * NT;
#pragma unroll
      for (int q = 0; q < R; ++q) a[i * R + q] = sbuf[spad(j + q * (N2 / R))];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * NT;
      const int k = j & (Ns - 1);
      if constexpr (Ns > 1) {
#pragma unroll
        for (int q = 1; q < R; ++q) a[i * R + q] = cmul(a[i * R + q], tw[(q - 1) * Ns + k]);
      }
      dft<R>(&a[i * R]);
      const int base = (j - k) * R + k;
      if constexpr (PUSH_P > 1) {
        constexpr int C = (N2 + PUSH_P - 1) / PUSH_P;
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int k2 = base + q * Ns, owner = k2 / C;
          st_async_c64(mapa_shared(push.recv_l + (uint32_t)(push.r * C + k2 - owner * C) * sizeof(float2), owner),
                       a[i * R + q], mapa_shared(push.bar0_l, owner));
        }
      } else {
#pragma unroll
        for (int q = 0; q < R; ++q) sbuf[spad(base + q * Ns)] = a[i * R + q];
      }
    }
  }
  __syncthreads();
}

// The transpose of ssm_pass (decimation in frequency): it reads where
// ssm_pass writes, runs the same radix-R DFT (a symmetric matrix), applies
// the twiddles after it and writes where ssm_pass reads.  With unit-modulus
// twiddles, conj o (these passes in reverse order) o conj is the exact
// inverse of the forward passes, up to the factor N2.
// LAST (the pass with Ns = 1, run last): the conjugation completes the
// inverse, then the Kerr step on the thread's 16 samples.
template <int LOGN2, int LOGNS, int LOGR, bool LAST>
__device__ __forceinline__ void ssm_pass_dif(float2* sbuf, const float2* __restrict__ stw, float c, int t,
                                             bool active) {
  constexpr int N2 = 1 << LOGN2, R = 1 << LOGR, Ns = 1 << LOGNS, NT = N2 / kSsmE, NB = kSsmE / R;
  const float2* __restrict__ tw = stw + ssm_stage_offset(LOGN2, LOGNS);
  float2 a[kSsmE];
  if (active) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * NT;
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int q = 0; q < R; ++q) a[i * R + q] = sbuf[spad(base + q * Ns)];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * NT;
      const int k = j & (Ns - 1);
      dft<R>(&a[i * R]);
      if constexpr (Ns > 1) {
#pragma unroll
        for (int q = 1; q < R; ++q) a[i * R + q] = cmul(a[i * R + q], tw[(q - 1) * Ns + k]);
      }
    }
    if constexpr (LAST) {
      static_assert(LOGNS == 0, "the last inverse pass is the one with Ns = 1");
#pragma unroll
      for (int q = 0; q < kSsmE; ++q) a[q] = make_float2(a[q].x, -a[q].y);
      if (c != 0.f) tile_kerr<kSsmE>(a, c);
    }
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int j = t + i * NT;
#pragma unroll
      for (int q = 0; q < R; ++q) sbuf[spad(j + q * (N2 / R))] = a[i * R + q];
    }
  }
  __syncthreads();
}

// Pass list of the local transform: pass 0 has radix 2^(LOGN2 % 4) (16 when
// LOGN2 % 4 == 0), every later pass radix 16.
__host__ __device__ constexpr int ssm_first_logr(int logn2) { return (logn2 % 4) != 0 ? (logn2 % 4) : 4; }
__host__ __device__ constexpr int ssm_pass_logns(int logn2, int idx) {
  return idx == 0 ? 0 : ssm_first_logr(logn2) + 4 * (idx - 1);
}
__host__ __device__ constexpr int ssm_pass_logr(int logn2, int idx) { return idx == 0 ? ssm_first_logr(logn2) : 4; }
__host__ __device__ constexpr int ssm_npass(int logn2) { return 1 + (logn2 - ssm_first_logr(logn2)) / 4; }

// Forward local transform: passes 0 .. npass-1 (the last one may push).
template <int LOGN2, int IDX, int PUSH_P = 0>
__device__ __forceinline__ void ssm_local_fft(float2* sbuf, const float2* stw, int t, bool active,
                                              const SsmPush& push = SsmPush{0u, 0u, 0}) {
  if constexpr (IDX < ssm_npass(LOGN2)) {
    constexpr bool last = IDX + 1 == ssm_npass(LOGN2);
    ssm_pass<LOGN2, ssm_pass_logns(LOGN2, IDX), ssm_pass_logr(LOGN2, IDX), last ? PUSH_P : 0>(sbuf, stw, t, active,
                                                                                              push);
    ssm_local_fft<LOGN2, IDX + 1, PUSH_P>(sbuf, stw, t, active, push);
  }
}

// Inverse local transform (on conjugated data): the transposed passes
// npass-1 .. 0, Kerr fused into pass 0.
template <int LOGN2, int IDX>
__device__ __forceinline__ void ssm_local_ifft(float2* sbuf, const float2* stw, float c, int t, bool active) {
  if constexpr (IDX >= 0) {
    ssm_pass_dif<LOGN2, ssm_pass_logns(LOGN2, IDX), ssm_pass_logr(LOGN2, IDX), IDX == 0>(sbuf, stw, c, t, active);
    ssm_local_ifft<LOGN2, IDX - 1>(sbuf, stw, c, t, active);
  }
}

template <int P>
__device__ __forceinline__ void cluster_barrier(cg::cluster_group& cl) {
  if constexpr (P > 1) cl.sync();
  else __syncthreads();
}

// Chunking of the N2 frequencies k2 among the P blocks of a cluster: block q
// owns k2 in [q C, q C + c_q) with C = ceil(N2 / P), so for P = 3, 6, 12 (a
// factor 3 in n) the last chunk is shorter.
template <int LOGN2, int P>
struct SsmChunk {
  static constexpr int N2 = 1 << LOGN2, C = (N2 + P - 1) / P;
  __device__ static int size(int q) { return q < P - 1 ? C : N2 - (P - 1) * C; }
};

// Spectral step across the cluster (see file comment, step 2).  Data move
// by asynchronous remote stores (st.async) that count their bytes on the
// receiver's mbarrier, so each block waits only for the data it needs: no
// cluster-wide barrier per step.
//  * bars[0] completes when this block's receive buffer holds all P chunks;
//  * bars[1] completes when all N2 results for this block have arrived.
// The ordering needs no further synchronisation: a block pushes results into
// block r's chunk q only after receiving that chunk from r (so r has read it),
// and r pushes its next spectrum only after all results of this step arrived
// (so every owner has finished reading its receive buffer).
template <int LOGN2, int P>
__device__ __forceinline__ bool ssm_middle(float2* sbuf, float2* recv, uint64_t* bars, uint32_t phase, int r, int b,
                                           const SsmStep& st, const SsmParams& p, bool first) {
  constexpr int N2 = 1 << LOGN2, NT = N2 / kSsmE, C = SsmChunk<LOGN2, P>::C, NK = (C + NT - 1) / NT;
  const int t = threadIdx.x;
  const int cr = SsmChunk<LOGN2, P>::size(r);  // frequencies this block owns
  bool ok = true;
  // The step's spectral values and the cluster twiddles of this thread's
  // frequencies are fetched from global memory first, so that their latency
  // overlaps the exchange below; with more than 16 twiddles per thread
  // (P = 12) the twiddles are loaded where they are used instead.
  constexpr bool kTwEarly = NK * (P - 1) <= 16;
  const float2* __restrict__ H = p.tabs[st.tab];
  const uint32_t* __restrict__ HL = p.tabs_lo[st.tab];
  const float hl_scale = p.tabs_lo_scale[st.tab];
  float2 hv[NK][P], wv[kTwEarly ? NK : 1][P > 1 ? P - 1 : 1];
  uint32_t hl[NK][P];
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int kk = t + i * NT, k2 = r * C + (kk < cr ? kk : 0);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      hv[i][k1] = __ldg(&H[k2 + N2 * k1]);
      hl[i][k1] = __ldg(&HL[k2 + N2 * k1]);
    }
    if constexpr (kTwEarly) {
#pragma unroll
      for (int q = 1; q < P; ++q) wv[i][q - 1] = __ldg(&p.twiddle[(q - 1) * N2 + k2]);
    }
  }
  if constexpr (P > 1) {
    // the forward transform's last pass has pushed this block's spectrum to the
    // owners (possibly before this expect_tx: the phase cannot complete before
    // this arrival, and the transaction count may go transiently negative)
    if (t == 0) {
      mbar_arrive_expect_tx(&bars[0], (uint32_t)(P * cr) * sizeof(float2));
      mbar_arrive_expect_tx(&bars[1], N2 * sizeof(float2));
    }
    ok = mbar_wait_cluster_bounded(&bars[0], phase, 1 << 20);
  }
  const float2* __restrict__ HN = st.noise_tab >= 0 ? p.tabs[st.noise_tab] : nullptr;
  const bool noise = st.noise_tab > -2;
  const float flat = 1.0f / (float)p.n;
  float sc = st.scale;
  if (first && p.wave_scale) {
    const float w = p.wave_scale[b];
    sc *= p.wave_mode == 1 ? sqrtf(w) : p.wave_mode == 2 ? rsqrtf(w) : w;
  }
  const uint32_t bar1_l = smem_u32(&bars[1]);
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    const int kk = t + i * NT, k2 = r * C + kk;
    if (NK * NT > C && kk >= cr) break;
    const int iw = kTwEarly ? i : 0;
    if constexpr (!kTwEarly) {
#pragma unroll
      for (int q = 1; q < P; ++q) wv[0][q - 1] = __ldg(&p.twiddle[(q - 1) * N2 + k2]);
    }
    float2 a[P];
#pragma unroll
    for (int q = 0; q < P; ++q) a[q] = P > 1 ? recv[q * C + kk] : sbuf[spad(k2)];
#pragma unroll
    for (int q = 1; q < P; ++q) a[q] = cmul(a[q], wv[iw][q - 1]);
    dft<P>(a);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      const int k = k2 + N2 * k1;
      float2 A = cmul_hl(a[k1], hv[i][k1], tail_h2(hl[i][k1], hl_scale));
      A = make_float2(A.x * sc, A.y * sc);
      if (noise) {
        const float2 g = ase_normal((uint32_t)k, (uint32_t)b, (uint32_t)st.span, p.counter, p.seed_lo, p.seed_hi);
        const float2 hn = HN ? __ldg(&HN[k]) : make_float2(flat, 0.f);
        A = cadd(A, cmul(hn, make_float2(g.x * p.noise_std, g.y * p.noise_std)));
      }
      a[k1] = make_float2(A.x, -A.y);
    }
    dft<P>(a);
    // Results go out as soon as they are formed: to block q's own slot of
    // the local sequence (remote store counted on its bars[1]), or in place.
    if constexpr (P > 1) {
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const float2 o = q == 0 ? a[0] : cmul(a[q], wv[iw][q - 1]);
        const uint32_t dst = mapa_shared(smem_u32(sbuf), q), rbar = mapa_shared(bar1_l, q);
        st_async_c64(dst + (uint32_t)spad(r * C + kk) * sizeof(float2), o, rbar);
      }
    } else {
      sbuf[spad(kk)] = a[0];
    }
  }
  if constexpr (P > 1) {
    ok = mbar_wait_cluster_bounded(&bars[1], phase, 1 << 20) && ok;
  } else {
    __syncthreads();
  }
  return ok;
}

template <int LOGN2, int P>
__global__ void __launch_bounds__((1 << LOGN2) / kSsmE, (512 / ((1 << LOGN2) / kSsmE)) > 1 ? (512 / ((1 << LOGN2) / kSsmE)) : 1) ssm_kernel(const __grid_constant__ SsmParams p) {
  constexpr int N2 = 1 << LOGN2, NT = N2 / kSsmE;
  extern __shared__ __align__(16) float2 sbuf[];  // [spad(N2)] data, then the local-pass twiddles
  constexpr int NTW = ssm_stage_offset(LOGN2, LOGN2);
  float2* stw = sbuf + N2 + N2 / 16;
  float2* recv = stw + NTW;  // [P][C] receive buffer of the cluster exchange (P > 1)
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ int stop;
  cg::cluster_group cl = cg::this_cluster();
  const int r = (int)cl.block_rank();
  const int b = blockIdx.x / P;
  const int t = threadIdx.x;
  const long long n = p.n;
  const float2* __restrict__ xin = p.x + (long long)b * n;
  for (int m2 = t; m2 < N2; m2 += NT) {
    float2 v = xin[r + (long long)P * m2];
    if (p.c_pre != 0.f) v = kerr_rotate_precise<true>(v, p.c_pre);
    sbuf[spad(m2)] = v;
  }
  for (int i = t; i < NTW; i += NT) stw[i] = p.twiddle[(P - 1) * N2 + i];
  if (t == 0) {
    stop = 0;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  cluster_barrier<P>(cl);  // every block of the cluster is running (barriers initialised) before remote access
  const SsmPush push{smem_u32(recv), smem_u32(&bars[0]), r};
  for (int s = 0; s < p.nsteps; ++s) {
    const SsmStep st = p.steps[s];
    ssm_local_fft<LOGN2, 0, P>(sbuf, stw, t, true, push);
    if (!ssm_middle<LOGN2, P>(sbuf, recv, bars, (uint32_t)(s & 1), r, b, st, p, s == 0)) stop = 1;
    ssm_local_ifft<LOGN2, ssm_npass(LOGN2) - 1>(sbuf, stw, st.c, t, true);  // its barriers make `stop` visible
    if (stop) break;
  }
  cluster_barrier<P>(cl);  // no block leaves while a peer may still store into it
  float2* __restrict__ yout = p.y + (long long)b * n;
  for (int m2 = t; m2 < N2; m2 += NT) yout[r + (long long)P * m2] = sbuf[spad(m2)];
}

template <int LOGN2, int P>
cudaError_t launch_one(const SsmParams& p, cudaStream_t st) {
  constexpr int N2 = 1 << LOGN2, NT = N2 / kSsmE;
  const size_t smem = sizeof(float2) * (size_t)(N2 + N2 / 16 + ssm_stage_offset(LOGN2, LOGN2) +
                                                 (P > 1 ? P * SsmChunk<LOGN2, P>::C : 0));
  auto kern = ssm_kernel<LOGN2, P>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (P > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(p.batch * P));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = P;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

}  // namespace ldbp
