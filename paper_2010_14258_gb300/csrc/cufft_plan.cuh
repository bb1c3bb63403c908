// Cached cuFFT plans of the library-FFT paths (batched C2C, contiguous rows).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

namespace ldbp {

// Plan of `batch` contiguous length-n C2C transforms, created on the first call
// for (device, stream, n, batch) and bound to `st`.  Keying by stream gives
// every stream its own cuFFT work area, so calls on different streams never
// share one.
int cufft_plan(long long n, int batch, cudaStream_t st, cufftHandle* out);

}  // namespace ldbp
