// Host side of the core SVD (Phase I on the core and H_r, Sec. 3.1 / 3.2):
// shared-memory sizing, the choice of cluster size, and the launches by padded
// rank.  The kernels are in svd_kernels.cuh; each rank's launch is
// instantiated in one of the k_svd_ranks_*.cu files, so that they compile in
// parallel.
#include <mutex>

#include "svd_kernels.cuh"

namespace ircur {

extern template cudaError_t svd_launch_r<1>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<1>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<2>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<2>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<3>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<3>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<4>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<4>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<5>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<5>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<6>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<6>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<7>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<7>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<8>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<8>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<9>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<9>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<10>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<10>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<12>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<12>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<16>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<16>(const BatchLaunch&, cudaStream_t);
extern template cudaError_t svd_launch_r<20>(const IterDesc&, cudaStream_t);
extern template cudaError_t svd_launch_batch_r<20>(const BatchLaunch&, cudaStream_t);

cudaError_t launch_sigma(const float* Tm, int r, int Rpad, float* sigma, cudaStream_t s) {
  switch (Rpad) {
#define IRCUR_SIGMA_CASE(RR) \
  case RR:                   \
    sigma_kernel<RR><<<1, 32, 0, s>>>(Tm, r, sigma); \
    break;
    IRCUR_SIGMA_CASE(1)
    IRCUR_SIGMA_CASE(2)
    IRCUR_SIGMA_CASE(3)
    IRCUR_SIGMA_CASE(4)
    IRCUR_SIGMA_CASE(5)
    IRCUR_SIGMA_CASE(6)
    IRCUR_SIGMA_CASE(7)
    IRCUR_SIGMA_CASE(8)
    IRCUR_SIGMA_CASE(9)
    IRCUR_SIGMA_CASE(10)
    IRCUR_SIGMA_CASE(12)
    IRCUR_SIGMA_CASE(16)
    IRCUR_SIGMA_CASE(20)
#undef IRCUR_SIGMA_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side

size_t svd_smem_bytes(int nI, int nJ, int Rpad, int nc) {
  const SvdGeom g = svd_geom(nI, nJ, Rpad, nc);
  return g.total > sizeof(SamplerSmem) ? g.total : sizeof(SamplerSmem);
}

bool svd_fits(int nI, int nJ, int Rpad, int nc) { return svd_smem_bytes(nI, nJ, Rpad, nc) <= 227 * 1024; }

// Whether the device runs clusters of 16 CTAs (a non-portable size) of the
// core SVD in its largest configuration (227 KB of shared memory per CTA):
// asked once per device.
static bool cluster16_ok() {
  static std::mutex mu;
  static signed char known[64];  // 0: not asked yet, 1: yes, -1: no
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (known[dev] == 0) known[dev] = svd_cluster16_capacity() > 0 ? 1 : -1;
  return known[dev] > 0;
}

// Cluster size of the core SVD: one CTA where the caller asked for it and the
// whole core fits one SM; 8 CTAs where the caller asked for them and the slabs
// of 8 fit; else 16 CTAs where the device runs clusters of 16 (half the slab
// work per CTA for one more level of the exchange), else 8.
// 0: no form fits.
int svd_cluster_size(int nI, int nJ, int Rpad, int svd_form) {
  if (svd_form == IRCUR_SVD_ONE_CTA && svd_fits(nI, nJ, Rpad, 1)) return 1;
  if (svd_form == IRCUR_SVD_CLUSTER8 && svd_fits(nI, nJ, Rpad, kSvdCluster)) return kSvdCluster;
  if (svd_fits(nI, nJ, Rpad, 16) && cluster16_ok()) return 16;
  if (svd_fits(nI, nJ, Rpad, kSvdCluster)) return kSvdCluster;
  return 0;
}

bool svd_shape_ok(int nI, int nJ, int Rpad, int svd_form) {
  if (svd_form == IRCUR_SVD_ONE_CTA && svd_fits(nI, nJ, Rpad, 1)) return true;
  return svd_fits(nI, nJ, Rpad, kSvdCluster) || svd_fits(nI, nJ, Rpad, 16);
}

cudaError_t launch_svd_batch(const BatchLaunch& b, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return svd_launch_batch_r<1>(b, s);
    case 2: return svd_launch_batch_r<2>(b, s);
    case 3: return svd_launch_batch_r<3>(b, s);
    case 4: return svd_launch_batch_r<4>(b, s);
    case 5: return svd_launch_batch_r<5>(b, s);
    case 6: return svd_launch_batch_r<6>(b, s);
    case 7: return svd_launch_batch_r<7>(b, s);
    case 8: return svd_launch_batch_r<8>(b, s);
    case 9: return svd_launch_batch_r<9>(b, s);
    case 10: return svd_launch_batch_r<10>(b, s);
    case 12: return svd_launch_batch_r<12>(b, s);
    case 16: return svd_launch_batch_r<16>(b, s);
    case 20: return svd_launch_batch_r<20>(b, s);
    default: return cudaErrorInvalidValue;
  }
}

// Batched IRCUR-R: the look-ahead draws (roles 1 and 2 of a core-SVD launch)
// as a launch of their own, one CTA per (instance, axis), so that a batch's
// core-SVD grid carries no cluster that only one CTA of works in.  The
// iteration k comes from the instance's state: the launch must end before the
// panel pass of the same iteration advances it.
__global__ void __launch_bounds__(512) sample_ahead_batch_kernel(const IterDesc* __restrict__ ds) {
  __shared__ SamplerSmem S;
  const IterDesc& d = ds[blockIdx.x];
  const State* st = d.st;
  if (st->done || st->status) return;
  svd_sample_ahead(d, st->k, (int)blockIdx.y, S);
}

cudaError_t launch_sample_ahead_batch(const IterDesc* ds, int count, cudaStream_t s) {
  sample_ahead_batch_kernel<<<dim3((unsigned)count, 2, 1), 512, 0, s>>>(ds);
  return cudaGetLastError();
}

cudaError_t launch_svd(const IterDesc& d, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return svd_launch_r<1>(d, s);
    case 2: return svd_launch_r<2>(d, s);
    case 3: return svd_launch_r<3>(d, s);
    case 4: return svd_launch_r<4>(d, s);
    case 5: return svd_launch_r<5>(d, s);
    case 6: return svd_launch_r<6>(d, s);
    case 7: return svd_launch_r<7>(d, s);
    case 8: return svd_launch_r<8>(d, s);
    case 9: return svd_launch_r<9>(d, s);
    case 10: return svd_launch_r<10>(d, s);
    case 12: return svd_launch_r<12>(d, s);
    case 16: return svd_launch_r<16>(d, s);
    case 20: return svd_launch_r<20>(d, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ircur
