// Instantiation of the core-SVD launches (svd_kernels.cuh) for padded rank 12.
#include "svd_kernels.cuh"

namespace ircur {

template cudaError_t svd_launch_r<12>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<12>(const BatchLaunch&, cudaStream_t);

}  // namespace ircur
