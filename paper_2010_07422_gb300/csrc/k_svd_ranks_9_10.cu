// Instantiation of the core-SVD launches (svd_kernels.cuh) for padded ranks 9, 10.
#include "svd_kernels.cuh"

namespace ircur {

template cudaError_t svd_launch_r<9>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<9>(const BatchLaunch&, cudaStream_t);
template cudaError_t svd_launch_r<10>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<10>(const BatchLaunch&, cudaStream_t);

}  // namespace ircur
