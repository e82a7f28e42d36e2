// Instantiation of the core-SVD launches (svd_kernels.cuh) for padded rank 20.
#include "svd_kernels.cuh"

namespace ircur {

template cudaError_t svd_launch_r<20>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<20>(const BatchLaunch&, cudaStream_t);

}  // namespace ircur
