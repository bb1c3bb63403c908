// Instances of the split-step kernel with cluster size 4.
#include "ssm_kernel.cuh"

namespace ldbp {
template cudaError_t launch_one<11, 4>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<12, 4>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<13, 4>(const SsmParams& p, cudaStream_t st);
}  // namespace ldbp
