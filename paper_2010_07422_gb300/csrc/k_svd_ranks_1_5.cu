// Instantiation of the core-SVD launches (svd_kernels.cuh) for padded ranks 1, 2, 3, 4, 5.
#include "svd_kernels.cuh"

namespace ircur {

template cudaError_t svd_launch_r<1>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<1>(const BatchLaunch&, cudaStream_t);
template cudaError_t svd_launch_r<2>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<2>(const BatchLaunch&, cudaStream_t);
template cudaError_t svd_launch_r<3>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<3>(const BatchLaunch&, cudaStream_t);
template cudaError_t svd_launch_r<4>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<4>(const BatchLaunch&, cudaStream_t);
template cudaError_t svd_launch_r<5>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<5>(const BatchLaunch&, cudaStream_t);

}  // namespace ircur
