// Instances of the split-step kernel with cluster size 16.
#include "ssm_kernel.cuh"

namespace ldbp {
template cudaError_t launch_one<11, 16>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<12, 16>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<13, 16>(const SsmParams& p, cudaStream_t st);
}  // namespace ldbp
