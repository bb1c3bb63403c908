// Shared device/host helpers of the GB300 split-step library (sm_103a only).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ldbp.h"

namespace ldbp {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define LDBP_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return ::ldbp::cuda_fail(_e, #expr); \
  } while (0)

// Device-side status word: kernels never trap; a bounded wait that runs out or
// a detected inconsistency records a code here and the kernel returns.
extern __device__ int g_device_status;
enum DeviceStatus : int { kDevOk = 0, kDevTimeout = 1, kDevBadArg = 2 };

__device__ __forceinline__ void device_flag(int code) { atomicCAS(&g_device_status, 0, code); }

// ---------------------------------------------------------------- complex
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * (h + l): product with a constant held as a float head h and a small
// tail l; the tail enters below the rounding of the head products.
__device__ __forceinline__ float2 cmul_hl(float2 a, float2 h, float2 l) {
  return make_float2(fmaf(a.x, h.x, fmaf(-a.y, h.y, fmaf(a.x, l.x, -a.y * l.y))),
                     fmaf(a.x, h.y, fmaf(a.y, h.x, fmaf(a.x, l.y, a.y * l.x))));
}
// Tail stored as half2 bits in units of `scale`.
__device__ __forceinline__ float2 tail_h2(uint32_t bits, float scale) {
  __half2 q;
  memcpy(&q, &bits, sizeof(q));
  const float2 f = __half22float2(q);
  return make_float2(f.x * scale, f.y * scale);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cfma(float2 h, float2 s, float2 acc) {  // acc + h*s
  acc.x = fmaf(h.x, s.x, acc.x);
  acc.x = fmaf(-h.y, s.y, acc.x);
  acc.y = fmaf(h.x, s.y, acc.y);
  acc.y = fmaf(h.y, s.x, acc.y);
  return acc;
}

// Kerr rotation x * exp(j c |x|^2) (the nonlinear step of the split-step method).
// __sincosf runs on the special-function unit; its absolute error is about
// 2^-21 for |phase| <= pi, the regime of fiber nonlinearity per step.
__device__ __forceinline__ float2 kerr_rotate(float2 v, float c) {
  float p = fmaf(v.x, v.x, v.y * v.y);
  float s, co;
  __sincosf(c * p, &s, &co);
  return make_float2(fmaf(v.x, co, -v.y * s), fmaf(v.x, s, v.y * co));
}

// exp(j phi) for the Kerr rotation, accurate to a few FP32 ulps for any phi
// with |phi| < 2^21.  Cody-Waite reduction by pi/2 (pi/2 split into a float
// head and tail), then Taylor polynomials of sin and cos on |r| <= pi/4
// (truncation below 2e-9), then the quadrant is restored by swapping and
// negating.  `reduce = false` skips the reduction; it is exact only for
// |phi| <= pi/4 and gives bit-identical results there.
template <bool reduce>
__device__ __forceinline__ float2 expj(float phi) {
  float r = phi;
  int q = 0;
  if constexpr (reduce) {
    const float kMagic = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer
    const float t = fmaf(phi, 0.636619772367581343f, kMagic);
    q = __float_as_int(t) - __float_as_int(kMagic);
    const float qf = t - kMagic;
    r = fmaf(-qf, 1.57079637050628662f, r);
    r = fmaf(-qf, -4.37113900018624283e-8f, r);
  }
  const float r2 = r * r;
  float s = fmaf(r2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);
  s = fmaf(r2, s, 8.33333333333333333e-3f);
  s = fmaf(r2, s, -1.66666666666666667e-1f);
  s = fmaf(r2 * r, s, r);
  float c = fmaf(r2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);
  c = fmaf(r2, c, -1.38888888888888889e-3f);
  c = fmaf(r2, c, 4.16666666666666667e-2f);
  c = fmaf(r2, c, -0.5f);
  c = fmaf(r2, c, 1.0f);
  if constexpr (reduce) {
    const float sw = (q & 1) ? c : s;
    const float cw = (q & 1) ? s : c;
    s = __int_as_float(__float_as_int(sw) ^ ((q & 2) << 30));
    c = __int_as_float(__float_as_int(cw) ^ (((q + 1) & 2) << 30));
  }
  return make_float2(c, s);
}

// Kerr rotation with the accurate exp(j phi); see expj.
template <bool reduce>
__device__ __forceinline__ float2 kerr_rotate_precise(float2 v, float c) {
  const float2 e = expj<reduce>(c * fmaf(v.x, v.x, v.y * v.y));
  return make_float2(fmaf(v.x, e.x, -v.y * e.y), fmaf(v.x, e.y, v.y * e.x));
}

// ---------------------------------------------------------------- async copy
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; returns false (and flags a timeout) when
// the iteration limit runs out.  try_wait itself suspends for a bounded time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit = 1 << 22) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  device_flag(kDevTimeout);
  return false;
}
// Arrive (no transaction bytes) with release semantics at CTA scope.
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait with acquire semantics at cluster scope (data written by peer blocks
// through st.async is visible after it returns true).
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t parity, int limit = 1 << 22) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait_cluster(bar, parity)) return true;
  device_flag(kDevTimeout);
  return false;
}
// Shared-memory address of the same variable in block `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t local_addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
  return r;
}
// Asynchronous remote store of one complex value into a peer block's shared
// memory; the peer's mbarrier `rbar` counts the 8 bytes on arrival.
__device__ __forceinline__ void st_async_c64(uint32_t raddr, float2 v, uint32_t rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
               "f"(v.x), "f"(v.y), "r"(rbar)
               : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// 1-D bulk copy shared -> global (TMA engine), tracked by the bulk async-group.
__device__ __forceinline__ void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(smem_u32(src_smem)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__host__ __device__ __forceinline__ bool aligned16(const void* p) {
  return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

}  // namespace ldbp
