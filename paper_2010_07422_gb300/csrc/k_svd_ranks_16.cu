// Instantiation of the core-SVD launches (svd_kernels.cuh) for padded rank 16,
// and the query of the device's capacity for clusters of 16 CTAs.
#include "svd_kernels.cuh"

namespace ircur {

template cudaError_t svd_launch_r<16>(const IterDesc&, cudaStream_t);
template cudaError_t svd_launch_batch_r<16>(const BatchLaunch&, cudaStream_t);

// Clusters of 16 CTAs of the R = 16 kernel with 227 KB of shared memory each
// that the current device holds at once (0: none, or the query failed).
int svd_cluster16_capacity() {
  auto kernel = csvd_kernel<16>;
  const int smem = 227 * 1024;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(16, 1, 1);
  cfg.blockDim = dim3(kSvdThreadsCl, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace ircur
