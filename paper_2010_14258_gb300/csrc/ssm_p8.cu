// Instances of the split-step kernel with cluster size 8.
#include "ssm_kernel.cuh"

namespace ldbp {
template cudaError_t launch_one<11, 8>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<12, 8>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<13, 8>(const SsmParams& p, cudaStream_t st);
}  // namespace ldbp
