// Instances of the split-step kernel with cluster size 3 (n = 3 * 2^k grids).
#include "ssm_kernel.cuh"

namespace ldbp {
template cudaError_t launch_one<9, 3>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<10, 3>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<11, 3>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<12, 3>(const SsmParams& p, cudaStream_t st);
}  // namespace ldbp
