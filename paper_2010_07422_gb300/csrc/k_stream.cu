// Streaming extension: new columns of D against the final CUR model of a
// solve.  Alg. 1 reads a column only through its entries on the rows I (its
// entry of R is d_I - S_I) and extends it to every row by L = C U^+ R, so a
// new column (a new frame of a video, Sec. 4.2) can go through Phase I / Phase
// II with the final iterate's C and U^+ held fixed; the paper leaves this step
// implicit.  With the solver's factors A = C X T^{-1} (n1 x R) and Y (|I| x R,
// the last core SVD's left basis), C U^+ r = A (Y^T r).  Per new column d,
// from L_0 = 0:
//   for t < iters:  zeta_t = gamma^t zeta_0 (repeated FP64 multiplication)
//     r = d_I - T_{zeta_t}(d_I - [L_t]_I)   (panel_value, as in the pass)
//     b = Y^T r,   [L_{t+1}]_I = A(I,:) b
//   L = A b,  S = T_{zeta_iters}(d - L).
// stream_fit_kernel: one warp per column, lanes over the rows of I (up to 16
// per lane), A(I,:) and Y staged in shared memory once per block; b goes to a
// small buffer.  stream_dense_kernel: L and S for every row of the new
// columns (row-major n1 x c blocks, as D is stored), bound by HBM like the
// reconstruction.
#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

constexpr int kStreamRowsPerLane = 16;  // |I| <= 512
constexpr int kStreamWarps = 8;

template <int R>
__global__ void __launch_bounds__(32 * kStreamWarps) stream_fit_kernel(
    const float* __restrict__ A, const int* __restrict__ I, const float* __restrict__ Y, int m,
    const float* __restrict__ Dn, int64_t ldDn, int64_t ncols, int iters, double zeta0, double gamma,
    float* __restrict__ bq) {
  extern __shared__ __align__(16) float sm[];
  float* AI = sm;                   // m x R: A(I,:)
  float* Ys = sm + (size_t)m * R;   // m x R: Y
  for (int q = threadIdx.x; q < m * R; q += blockDim.x) {
    const int a = q / R, t = q - a * R;
    AI[q] = A[(int64_t)I[a] * R + t];
    Ys[q] = Y[q];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * kStreamWarps + warp;
  if (col >= ncols) return;
  float dv[kStreamRowsPerLane];
#pragma unroll
  for (int j = 0; j < kStreamRowsPerLane; ++j) {
    const int a = lane + 32 * j;
    dv[j] = a < m ? Dn[(int64_t)I[a] * ldDn + col] : 0.f;
  }
  float b[R];
#pragma unroll
  for (int t = 0; t < R; ++t) b[t] = 0.f;
  double zeta = zeta0;
  for (int it = 0; it < iters; ++it) {
    const float z = (float)zeta;
    float acc[R];
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = 0.f;
#pragma unroll
    for (int j = 0; j < kStreamRowsPerLane; ++j) {
      const int a = lane + 32 * j;
      if (a < m) {
        const float l = lowrank_entry<R>(AI + (size_t)a * R, b);
        const float v = panel_value(dv[j], l, z);
#pragma unroll
        for (int t = 0; t < R; ++t) acc[t] = fmaf(Ys[(size_t)a * R + t], v, acc[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < R; ++t) b[t] = warp_sum(acc[t]);
    zeta = zeta * gamma;
  }
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < R; ++t) bq[col * R + t] = b[t];
  }
}

// 32 columns x 8 rows per block of 256 threads.
template <int R, bool WITH_S>
__global__ void __launch_bounds__(256) stream_dense_kernel(const float* __restrict__ A, const float* __restrict__ bq,
                                                           const float* __restrict__ Dn, int64_t ldDn, int64_t n1,
                                                           int64_t ncols, float zetaT, float* __restrict__ L,
                                                           int64_t ldL, float* __restrict__ S, int64_t ldS) {
  const int64_t col = (int64_t)blockIdx.y * 32 + (threadIdx.x & 31);
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= ncols || row >= n1) return;
  float a[R], bc[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    a[t] = A[row * R + t];
    bc[t] = bq[col * R + t];
  }
  const float l = lowrank_entry<R>(a, bc);
  L[row * ldL + col] = l;
  if (WITH_S) {
    const float x = Dn[row * ldDn + col] - l;
    S[row * ldS + col] = fabsf(x) > zetaT ? x : 0.f;
  }
}

template <int R>
static cudaError_t launch_stream_r(const float* A, const int* I, const float* Y, int m, int64_t n1, const float* Dn,
                                   int64_t ldDn, int64_t ncols, int iters, double zeta0, double gamma, float zetaT,
                                   float* bq, float* L, int64_t ldL, float* S, int64_t ldS, cudaStream_t s) {
  const size_t smem = (size_t)2 * m * R * 4;
  cudaError_t e = cudaFuncSetAttribute(stream_fit_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned fit_blocks = (unsigned)((ncols + kStreamWarps - 1) / kStreamWarps);
  stream_fit_kernel<R><<<fit_blocks, 32 * kStreamWarps, smem, s>>>(A, I, Y, m, Dn, ldDn, ncols, iters, zeta0,
                                                                    gamma, bq);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((n1 + 7) / 8), (unsigned)((ncols + 31) / 32), 1);
  if (S)
    stream_dense_kernel<R, true><<<grid, 256, 0, s>>>(A, bq, Dn, ldDn, n1, ncols, zetaT, L, ldL, S, ldS);
  else
    stream_dense_kernel<R, false><<<grid, 256, 0, s>>>(A, bq, Dn, ldDn, n1, ncols, zetaT, L, ldL, S, ldS);
  return cudaGetLastError();
}

cudaError_t launch_stream(const float* A, const int* I, const float* Y, int m, int Rpad, int64_t n1, const float* Dn,
                          int64_t ldDn, int64_t ncols, int iters, double zeta0, double gamma, float zetaT, float* bq,
                          float* L, int64_t ldL, float* S, int64_t ldS, cudaStream_t s) {
  if (m > 32 * kStreamRowsPerLane) return cudaErrorInvalidValue;
  switch (Rpad) {
#define IRCUR_STREAM_CASE(RR) \
  case RR:                    \
    return launch_stream_r<RR>(A, I, Y, m, n1, Dn, ldDn, ncols, iters, zeta0, gamma, zetaT, bq, L, ldL, S, ldS, s);
    IRCUR_STREAM_CASE(1)
    IRCUR_STREAM_CASE(2)
    IRCUR_STREAM_CASE(3)
    IRCUR_STREAM_CASE(4)
    IRCUR_STREAM_CASE(5)
    IRCUR_STREAM_CASE(6)
    IRCUR_STREAM_CASE(7)
    IRCUR_STREAM_CASE(8)
    IRCUR_STREAM_CASE(9)
    IRCUR_STREAM_CASE(10)
    IRCUR_STREAM_CASE(12)
    IRCUR_STREAM_CASE(16)
    IRCUR_STREAM_CASE(20)
#undef IRCUR_STREAM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ircur
