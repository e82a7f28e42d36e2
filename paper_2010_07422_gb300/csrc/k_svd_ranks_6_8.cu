// Instantiation of the core-SVD launches (svd_kernels.cuh) for padded ranks 6, 7, 8.
#include "svd_kernels.cuh"

namespace ircur {

template cudaError_t svd_launch_r<6>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<6>(const BatchLaunch&, cudaStream_t);
template cudaError_t svd_launch_r<7>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<7>(const BatchLaunch&, cudaStream_t);
template cudaError_t svd_launch_r<8>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<8>(const BatchLaunch&, cudaStream_t);

}  // namespace ircur
