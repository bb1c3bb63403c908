// Instances of the split-step kernel with cluster size 6 (n = 3 * 2^k grids).
#include "ssm_kernel.cuh"

namespace ldbp {
template cudaError_t launch_one<9, 6>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<10, 6>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<11, 6>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<12, 6>(const SsmParams& p, cudaStream_t st);
}  // namespace ldbp
