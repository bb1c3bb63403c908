// Instances of the split-step kernel with cluster size 1.
#include "ssm_kernel.cuh"

namespace ldbp {
template cudaError_t launch_one<9, 1>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<10, 1>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<11, 1>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<12, 1>(const SsmParams& p, cudaStream_t st);
template cudaError_t launch_one<13, 1>(const SsmParams& p, cudaStream_t st);
}  // namespace ldbp
