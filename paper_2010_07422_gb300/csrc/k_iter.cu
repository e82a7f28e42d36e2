// One IRCUR iteration (Alg. 1) on the GPU, in three kernels:
//   core_kernel  -- [D - S_{k+1}]_{I,J}: Phase I on the |I| x |J| block,
//   svd_kernel   -- H_r of the core and its pseudo-inverse (k_svd.cu),
//   pass_kernel  -- the fused panel passes and the stopping criterion.
//
// The iterate L_k = C_k U_k^+ R_k is never formed (Alg. 1); it is carried as
// the skinny factors A_k = C_k V_r Sigma_r^{-1} (n1 x r) and B_k = W_r^T R_k
// (r x n2), L_k = A_k B_k, so [L_k]_{I,:} and [L_k]_{:,J} (the two panel
// formulas of Sec. 3.2) are evaluated entry by entry as A_k(i,:) B_k(:,j).
// With U = W_r Sigma_r V_r^T the update C U^+ R factors as
// (C V_r Sigma_r^{-1})(W_r^T R): the column pass produces A_{k+1}, the row
// pass B_{k+1}.  Because C(I,:) = R(:,J) = core, L_{k+1}(I,:) = W_r W_r^T R
// and L_{k+1}(:,J) = C V_r V_r^T, so the stopping criterion of Sec. 3.3 is
// e = (||R - W_r W_r^T R||_F + ||C - C V_r V_r^T||_F) / (||D_{I,:}||_F + ||D_{:,J}||_F),
// each residual formed explicitly (no difference of squared norms).
#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

constexpr int kPassThreads = 128;
constexpr int kMaxQ = 16;  // column-pass register block: nJ <= 32 * kMaxQ

int pad_rank(int r) {
  if (r <= 10) return r;
  if (r <= 12) return 12;
  return 16;
}

// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(256) core_kernel(IterDesc d) {
  const State* st = d.st;
  if (st->done || st->status) return;
  const int k = st->k;
  const float zeta = (float)st->zeta;
  const int cur = k & 1;
  const int* I = d.I_all + (d.resample ? (int64_t)k * d.nI : 0);
  const int* J = d.J_all + (d.resample ? (int64_t)k * d.nJ : 0);
  const float* A = d.A[cur];
  const float* B = d.B[cur];
  for (int a = blockIdx.x; a < d.nI; a += gridDim.x) {
    const int ia = I[a];
    float arow[R];
#pragma unroll
    for (int t = 0; t < R; ++t) arow[t] = A[(int64_t)ia * R + t];
    const float* rowp = d.Prow ? d.Prow + (int64_t)a * d.ldPr : d.D + (int64_t)ia * d.ldD;
    for (int b = threadIdx.x; b < d.nJ; b += blockDim.x) {
      const int j = J[b];
      float bcol[R];
#pragma unroll
      for (int t = 0; t < R; ++t) bcol[t] = B[(int64_t)t * d.n2 + j];
      const float l = lowrank_entry<R>(arow, bcol);
      d.core[(int64_t)a * d.nJ + b] = panel_value(rowp[j], l, zeta);
    }
  }
}

// ---------------------------------------------------------------------------
// Row pass, one block per tile of rowTile consecutive columns j:
//   R_{k+1}(:,j) = D(I,j) - T_zeta(D(I,j) - A_k(I,:) B_k(:,j)),
//   B_{k+1}(:,j) = W_r^T R_{k+1}(:,j),
//   partial sums of ||R_{k+1}(:,j) - W_r B_{k+1}(:,j)||^2 and ||D(I,j)||^2.
// The |I| x rowTile tile is staged in shared memory by bulk copies (one per
// row of the panel, TMA engine) and overwritten in place with R_{k+1}, which
// the second sweep reads back for the explicit residual.
template <int R>
__device__ void row_pass(const IterDesc& d, int tile, int k, float zeta, unsigned char* smem, double* acc2) {
  const int nI = d.nI, TC = d.rowTile;
  const int cur = k & 1, nxt = cur ^ 1;
  const int* I = d.I_all + (d.resample ? (int64_t)k * nI : 0);
  float* tileS = reinterpret_cast<float*>(smem);                                // nI x TC
  float* AI = tileS + (size_t)nI * TC;                                          // nI x R
  float* Ws = AI + (size_t)nI * R;                                              // nI x R
  uint64_t* bar = reinterpret_cast<uint64_t*>(Ws + (size_t)nI * R);  // even float offset: 8-byte aligned
  const int64_t j0 = (int64_t)tile * TC;
  const int ncols = (int)((d.n2 - j0) < TC ? (d.n2 - j0) : TC);
  const float* A = d.A[cur];
  const float* rowsrc = d.Prow ? d.Prow : d.D;
  const int64_t ld = d.Prow ? d.ldPr : d.ldD;
  const bool bulk = d.rowBulk && ncols == TC;

  if (bulk && threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int q = threadIdx.x; q < nI * R; q += blockDim.x) {
    const int a = q / R, t = q - a * R;
    AI[q] = A[(int64_t)I[a] * R + t];
    Ws[q] = d.W[q];
  }
  __syncthreads();
  bool ok = true;
  if (bulk) {
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (unsigned)(nI * TC * 4));
    __syncwarp();
    if (threadIdx.x < 32) {
      for (int a = threadIdx.x; a < nI; a += 32) {
        const int64_t row = d.Prow ? a : I[a];
        bulk_g2s(tileS + (size_t)a * TC, rowsrc + row * ld + j0, (unsigned)(TC * 4), bar);
      }
    }
    ok = mbar_wait_bounded(bar, 0, d.spinLimit);
    if (!ok) {
      atomicExch(&d.st->status, (int)IRCUR_ETIMEOUT);
      mbar_wait_bounded(bar, 0, kSpinLimit);  // give copies in flight a second chance to land
    }
  } else {
    for (int a = 0; a < nI; ++a) {
      const int64_t row = d.Prow ? a : I[a];
      const float* src = rowsrc + row * ld + j0;
      for (int c = threadIdx.x; c < TC; c += blockDim.x) tileS[(size_t)a * TC + c] = c < ncols ? src[c] : 0.f;
    }
  }
  ok = __syncthreads_and(ok);
  if (!ok) return;

  const int jl = threadIdx.x;
  if (jl < ncols) {
    const int64_t j = j0 + jl;
    const float* B = d.B[cur];
    float bcol[R], bn[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      bcol[t] = B[(int64_t)t * d.n2 + j];
      bn[t] = 0.f;
    }
    float den = 0.f;
    for (int a = 0; a < nI; ++a) {
      float* cell = tileS + (size_t)a * TC + jl;
      const float dv = *cell;
      const float l = lowrank_entry<R>(AI + (size_t)a * R, bcol);
      const float v = panel_value(dv, l, zeta);
      *cell = v;
      den = fmaf(dv, dv, den);
#pragma unroll
      for (int t = 0; t < R; ++t) bn[t] = fmaf(Ws[(size_t)a * R + t], v, bn[t]);
    }
    float* Bn = d.B[nxt];
#pragma unroll
    for (int t = 0; t < R; ++t) Bn[(int64_t)t * d.n2 + j] = bn[t];
    float num = 0.f;
    for (int a = 0; a < nI; ++a) {
      const float v = tileS[(size_t)a * TC + jl];
      float w = 0.f;
#pragma unroll
      for (int t = 0; t < R; ++t) w = fmaf(Ws[(size_t)a * R + t], bn[t], w);
      const float rr = v - w;
      num = fmaf(rr, rr, num);
    }
    acc2[0] += (double)num;
    acc2[1] += (double)den;
  }
}

// Column pass, one warp per row i (rows strided over all column-pass warps):
//   C_{k+1}(i,:) = D(i,J) - T_zeta(D(i,J) - A_k(i,:) B_k(:,J)),
//   A_{k+1}(i,:) = C_{k+1}(i,:) V_r Sigma_r^{-1},
//   partial sums of ||C_{k+1}(i,:) - A_{k+1}(i,:) Sigma_r V_r^T||^2 and ||D(i,J)||^2.
// B_k(:,J), V_r Sigma_r^{-1} and V_r sit transposed in shared memory; a lane
// keeps its |J|/32 panel entries in registers.
template <int R>
__device__ void col_pass(const IterDesc& d, int cblock, int k, float zeta, unsigned char* smem, double* acc2) {
  const int nJ = d.nJ;
  const int cur = k & 1, nxt = cur ^ 1;
  const int* J = d.J_all + (d.resample ? (int64_t)k * nJ : 0);
  float* BJ = reinterpret_cast<float*>(smem);  // R x nJ
  float* VsT = BJ + (size_t)R * nJ;            // R x nJ
  float* VT = VsT + (size_t)R * nJ;            // R x nJ
  int* Js = reinterpret_cast<int*>(VT + (size_t)R * nJ);
  const float* B = d.B[cur];
  for (int q = threadIdx.x; q < R * nJ; q += blockDim.x) {
    const int t = q / nJ, b = q - t * nJ;
    BJ[q] = B[(int64_t)t * d.n2 + J[b]];
    VsT[q] = d.Vs[(size_t)b * R + t];
    VT[q] = d.V[(size_t)b * R + t];
  }
  for (int b = threadIdx.x; b < nJ; b += blockDim.x) Js[b] = J[b];
  float sig[R];
#pragma unroll
  for (int t = 0; t < R; ++t) sig[t] = d.sigma[t];
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int64_t gw = (int64_t)cblock * wpb + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)d.nColBlocks * wpb;
  const float* A = d.A[cur];
  float* An = d.A[nxt];
  double num_acc = 0.0, den_acc = 0.0;
  for (int64_t i = gw; i < d.n1; i += nw) {
    float arow[R];
#pragma unroll
    for (int t = 0; t < R; ++t) arow[t] = A[i * R + t];
    const float* src = d.Pcol ? d.Pcol + i * d.ldPc : d.D + i * d.ldD;
    float cv[kMaxQ];
    float an[R];
#pragma unroll
    for (int t = 0; t < R; ++t) an[t] = 0.f;
    float den = 0.f;
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) {
      const int b = lane + 32 * q;
      cv[q] = 0.f;
      if (b < nJ) {
        const float dv = d.Pcol ? src[b] : src[Js[b]];
        float bcol[R];
#pragma unroll
        for (int t = 0; t < R; ++t) bcol[t] = BJ[(size_t)t * nJ + b];
        const float v = panel_value(dv, lowrank_entry<R>(arow, bcol), zeta);
        cv[q] = v;
        den = fmaf(dv, dv, den);
#pragma unroll
        for (int t = 0; t < R; ++t) an[t] = fmaf(v, VsT[(size_t)t * nJ + b], an[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < R; ++t) an[t] = warp_sum(an[t]);
#pragma unroll
    for (int t = 0; t < R; ++t)
      if (lane == t) An[i * R + t] = an[t];
    float cs[R];
#pragma unroll
    for (int t = 0; t < R; ++t) cs[t] = an[t] * sig[t];
    float num = 0.f;
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) {
      const int b = lane + 32 * q;
      if (b < nJ) {
        float w = 0.f;
#pragma unroll
        for (int t = 0; t < R; ++t) w = fmaf(cs[t], VT[(size_t)t * nJ + b], w);
        const float rr = cv[q] - w;
        num = fmaf(rr, rr, num);
      }
    }
    num_acc += (double)num;
    den_acc += (double)den;
  }
  acc2[2] += num_acc;
  acc2[3] += den_acc;
}

// Fused row and column passes; the last block to finish reduces the
// per-block partial sums in a fixed order, evaluates e_{k+1}, advances k and
// zeta, and drives the graph's while-node (Alg. 1 loop "while e_k > epsilon").
template <int R>
__global__ void __launch_bounds__(kPassThreads) pass_kernel(IterDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  State* st = d.st;
  if (st->done || st->status) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->done = 1;
      if (d.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)d.cond, 0u);
    }
    return;
  }
  const int k = st->k;
  const float zeta = (float)st->zeta;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if ((int)blockIdx.x < d.nRowBlocks)
    row_pass<R>(d, blockIdx.x, k, zeta, smem, acc);
  else
    col_pass<R>(d, blockIdx.x - d.nRowBlocks, k, zeta, smem, acc);

  // block reduction of the four partial sums (fixed order)
  __shared__ double red[4][kPassThreads / 32];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kPassThreads / 32; ++w) s += red[threadIdx.x][w];
    d.partials[(size_t)blockIdx.x * 4 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // warp q sums partial q over all blocks (lane-strided, then a fixed tree)
  if (warp < 4) {
    double s = 0.0;
    const volatile double* pv = d.partials;
    for (unsigned b = lane; b < gridDim.x; b += 32) s += pv[(size_t)b * 4 + warp];
    s = warp_sum(s);
    if (lane == 0) red[warp][0] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double num = sqrt(red[0][0]) + sqrt(red[2][0]);
    const double den = sqrt(red[1][0]) + sqrt(red[3][0]);
    const double e = den > 0.0 ? num / den : 0.0;
    d.errs[k] = e;
    st->e = e;
    st->k = k + 1;
    st->zeta = st->zeta * d.gamma;
    st->counter = 0u;
    const int done = (e <= d.tol) || (k + 1 >= d.max_iter) || (st->status != 0);
    st->done = done;
    __threadfence();
    if (d.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)d.cond, done ? 0u : 1u);
  }
}

size_t pass_smem_bytes(int nI, int nJ, int Rpad, int rowTile) {
  const size_t row = (size_t)nI * rowTile * 4 + 2 * (size_t)nI * Rpad * 4 + 16 + 16;
  const size_t col = 3 * (size_t)Rpad * nJ * 4 + (size_t)nJ * 4 + 16;
  return row > col ? row : col;
}

cudaError_t launch_svd(const IterDesc& d, int Rpad, cudaStream_t s);

template <int R>
static cudaError_t launch_iter_r(const IterDesc& d, cudaStream_t s) {
  {
    int blocks = d.nI < 4 * kNumSMsHint ? d.nI : 4 * kNumSMsHint;
    core_kernel<R><<<blocks, 256, 0, s>>>(d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  {
    cudaError_t e = launch_svd(d, R, s);
    if (e != cudaSuccess) return e;
  }
  const size_t bytes = pass_smem_bytes(d.nI, d.nJ, R, d.rowTile);
  cudaError_t e = cudaFuncSetAttribute(pass_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  pass_kernel<R><<<d.nRowBlocks + d.nColBlocks, kPassThreads, bytes, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_iteration(const IterDesc& d, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_iter_r<1>(d, s);
    case 2: return launch_iter_r<2>(d, s);
    case 3: return launch_iter_r<3>(d, s);
    case 4: return launch_iter_r<4>(d, s);
    case 5: return launch_iter_r<5>(d, s);
    case 6: return launch_iter_r<6>(d, s);
    case 7: return launch_iter_r<7>(d, s);
    case 8: return launch_iter_r<8>(d, s);
    case 9: return launch_iter_r<9>(d, s);
    case 10: return launch_iter_r<10>(d, s);
    case 12: return launch_iter_r<12>(d, s);
    case 16: return launch_iter_r<16>(d, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ircur
