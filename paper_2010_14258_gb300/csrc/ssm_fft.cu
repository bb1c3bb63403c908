// Dispatch of the cluster-resident split-step kernel over (N2, P) and the
// choice of the cluster size (n = 2^k, or n = 3 * 2^k with P = 3, 6, 12).  The kernel instances live in ssm_p*.cu so that
// they compile in parallel.
#include "common.cuh"
#include "ssm.cuh"
#include "ssm_kernel.cuh"

namespace ldbp {

template <int LOGN2, int P>
cudaError_t launch_one(const SsmParams& p, cudaStream_t st);

#define LDBP_SSM_CASES(L)                          \
  case 1: return launch_one<L, 1>(p, st);          \
  case 2: return launch_one<L, 2>(p, st);          \
  case 4: return launch_one<L, 4>(p, st);          \
  case 8: return launch_one<L, 8>(p, st);          \
  case 16: return launch_one<L, 16>(p, st);        \
  default: return cudaErrorInvalidValue;

#define LDBP_SSM_CASES3(L)                         \
  case 3: return launch_one<L, 3>(p, st);          \
  case 6: return launch_one<L, 6>(p, st);          \
  case 12: return launch_one<L, 12>(p, st);        \
  default: return cudaErrorInvalidValue;

cudaError_t launch_ssm(const SsmParams& p, int P, int log_n2, cudaStream_t st) {
  if (P % 3 == 0) {
    switch (log_n2) {
      case 9: switch (P) { LDBP_SSM_CASES3(9) }
      case 10: switch (P) { LDBP_SSM_CASES3(10) }
      case 11: switch (P) { LDBP_SSM_CASES3(11) }
      case 12: switch (P) { LDBP_SSM_CASES3(12) }
      default: return cudaErrorInvalidValue;
    }
  }
  switch (log_n2) {
    case 9: return P == 1 ? launch_one<9, 1>(p, st) : cudaErrorInvalidValue;
    case 10: return P == 1 ? launch_one<10, 1>(p, st) : cudaErrorInvalidValue;
    case 11: switch (P) { LDBP_SSM_CASES(11) }
    case 12: switch (P) { LDBP_SSM_CASES(12) }
    case 13: switch (P) { LDBP_SSM_CASES(13) }
    default: return cudaErrorInvalidValue;
  }
}

long long ssm_twiddle_count(int P, int log_n2) {
  return (long long)(P - 1) * (1LL << log_n2) + ssm_stage_offset(log_n2, log_n2);
}

int ssm_choose_cluster(long long n, int batch, int sm_count, int* P, int* log_n2) {
  if (n % 3 == 0) {
    // n = 3 * 2^k: clusters of 3, 6 or 12 blocks over power-of-two blocks of
    // 2^9 .. 2^12 samples; blocks of at most 2048 samples while the cluster
    // allows, more blocks per waveform while the batch does not fill the GPU
    const long long m = n / 3;
    int k = 0;
    while ((1LL << k) < m) ++k;
    if ((1LL << k) != m) return -1;
    int p = 3, l = k;
    while (l > 11 && p < 12) p *= 2, --l;
    while (p < 12 && l - 1 >= 9 && (long long)batch * p < sm_count) p *= 2, --l;
    if (l < 9 || l > 12) return -1;
    *P = p;
    *log_n2 = l;
    return 0;
  }
  int logn = 0;
  while ((1LL << logn) < n) ++logn;
  if ((1LL << logn) != n || logn < kSsmMinLogN2 || logn > kSsmMaxLogN2 + 4) return -1;
  int p = 1;
  // blocks of at most 4096 samples (two or three blocks per SM) while the cluster allows
  while (logn - __builtin_ctz(p) > 12 && p < kSsmMaxCluster) p *= 2;
  if (logn - __builtin_ctz(p) > kSsmMaxLogN2) return -1;
  // more blocks per waveform while the batch alone does not fill the GPU
  while (p < 16 && logn - __builtin_ctz(p) - 1 >= 11 && (long long)batch * p < sm_count) p *= 2;
  *P = p;
  *log_n2 = logn - __builtin_ctz(p);
  return 0;
}

}  // namespace ldbp
