// One IRCUR iteration (Alg. 1) on the GPU, in three kernels:
//   core_kernel  -- [D - S_{k+1}]_{I,J}: Phase I on the |I| x |J| block,
//   svd_kernel   -- H_r of the core and its pseudo-inverse (k_svd.cu),
//   pass_kernel  -- the fused row- and column-panel passes and the stopping
//                   criterion.
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
    const float* rowp = d.rowSrc + (int64_t)(d.resample ? ia : a) * d.rowLd;
    for (int b = threadIdx.x; b < d.nJ; b += blockDim.x) {
      const int j = J[b];
      float bcol[R];
#pragma unroll
      for (int t = 0; t < R; ++t) bcol[t] = B[(int64_t)t * d.n2 + j];
      const float l = lowrank_entry<R>(arow, bcol);
      d.core[(int64_t)a * d.ldCore + b] = panel_value(rowp[j], l, zeta);
    }
  }
}

// ---------------------------------------------------------------------------
// One panel pass over a tile of kPanelCols consecutive panel columns.
//
// Row pass (COL = false): the panel is D(I,:) (m = |I| rows); for column j
//   R_{k+1}(:,j) = D(I,j) - T_zeta(D(I,j) - A_k(I,:) B_k(:,j)),
//   B_{k+1}(:,j) = Y^T R_{k+1}(:,j),
//   num += ||R_{k+1}(:,j) - Y B_{k+1}(:,j)||^2,  den += ||D(I,j)||^2.
// Column pass (COL = true): the panel is D(:,J)^T (m = |J| rows); for row i
//   C_{k+1}(i,:) = D(i,J) - T_zeta(D(i,J) - A_k(i,:) B_k(:,J)),
//   A_{k+1}(i,:) = C_{k+1}(i,:) X T^{-1},
//   num += ||C_{k+1}(i,:) - A_{k+1}(i,:) T X^T||^2,  den += ||D(i,J)||^2.
// Both are the same computation on a row-major m x n panel with
//   side = A_k(I,:) | B_k(:,J)^T (m x R), vec = B_k(:,j) | A_k(i,:)^T,
//   proj = Y | X T^{-1},  recon = Y | X T^T  (U^+ = X T^{-1} Y^T, see k_svd.cu).
// The m x kPanelCols tile is staged in shared memory by one bulk copy (TMA
// engine) per panel row, overwritten with D - S, and read back by the second
// sweep for the explicit residual.  kPanelSplit threads share a column, each
// sweeping a contiguous share of the rows; their partial projections are
// added in a fixed order.
template <int R, bool COL>
__device__ void panel_pass(const IterDesc& d, int tile, int k, float zeta, unsigned char* smem, double* acc2) {
  const int m = COL ? d.nJ : d.nI;
  const int64_t ncolsTotal = COL ? d.n1 : d.n2;
  const int cur = k & 1, nxt = cur ^ 1;
  const int* I = d.I_all + (d.resample ? (int64_t)k * d.nI : 0);
  const int* J = d.J_all + (d.resample ? (int64_t)k * d.nJ : 0);
  const int* map = COL ? J : I;
  const bool mapped = d.resample != 0;
  const float* src = COL ? d.colSrc : d.rowSrc;
  const int64_t ld = COL ? d.colLd : d.rowLd;

  float* tileS = reinterpret_cast<float*>(smem);           // m x kPanelCols
  float* side = tileS + (size_t)m * kPanelCols;             // m x R
  float* proj = side + (size_t)m * R;                       // m x R
  float* recon = COL ? proj + (size_t)m * R : proj;         // m x R (row pass: recon == proj)
  float* part = proj + (size_t)(COL ? 2 : 1) * m * R;       // kPanelSplit x kPanelCols x R
  // 8-byte aligned slot after the partial sums
  uintptr_t bp = reinterpret_cast<uintptr_t>(part + (size_t)kPanelSplit * kPanelCols * R);
  uint64_t* bar = reinterpret_cast<uint64_t*>((bp + 7) & ~(uintptr_t)7);

  const int64_t j0 = (int64_t)tile * kPanelCols;
  const int ncols = (int)((ncolsTotal - j0) < kPanelCols ? (ncolsTotal - j0) : kPanelCols);
  const bool bulk = (COL ? d.colBulk : d.rowBulk) && ncols == kPanelCols;

  if (bulk && threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (!COL) {
    const float* A = d.A[cur];
    for (int q = threadIdx.x; q < m * R; q += blockDim.x) {
      const int a = q / R, t = q - a * R;
      side[q] = A[(int64_t)I[a] * R + t];
      proj[q] = d.W[q];
    }
  } else {
    const float* B = d.B[cur];
    for (int q = threadIdx.x; q < m * R; q += blockDim.x) {
      const int b = q / R, t = q - b * R;
      side[q] = B[(int64_t)t * d.n2 + J[b]];
      proj[q] = d.Vs[q];
      recon[q] = d.V[q];
    }
  }
  __syncthreads();
  bool ok = true;
  if (bulk) {
    if (threadIdx.x == 0) mbar_arrive_expect_tx(bar, (unsigned)(m * kPanelCols * 4));
    __syncwarp();
    if (threadIdx.x < 32) {
      for (int a = threadIdx.x; a < m; a += 32) {
        const int64_t row = mapped ? map[a] : a;
        bulk_g2s(tileS + (size_t)a * kPanelCols, src + row * ld + j0, (unsigned)(kPanelCols * 4), bar);
      }
    }
    ok = mbar_wait_bounded(bar, 0, d.spinLimit);
    if (!ok) {
      atomicExch(&d.st->status, (int)IRCUR_ETIMEOUT);
      mbar_wait_bounded(bar, 0, kSpinLimit);  // let copies in flight land before the block exits
    }
  } else {
    for (int q = threadIdx.x; q < m * kPanelCols; q += blockDim.x) {
      const int a = q / kPanelCols, c = q - a * kPanelCols;
      const int64_t row = mapped ? map[a] : a;
      tileS[q] = c < ncols ? src[row * ld + j0 + c] : 0.f;
    }
  }
  ok = __syncthreads_and(ok);
  if (!ok) return;

  const int c = threadIdx.x % kPanelCols, h = threadIdx.x / kPanelCols;
  const int a0 = (int)((long long)h * m / kPanelSplit), a1 = (int)((long long)(h + 1) * m / kPanelSplit);
  const bool live = c < ncols;
  const int64_t j = j0 + c;
  float vec[R], acc[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    vec[t] = 0.f;
    acc[t] = 0.f;
  }
  if (live) {
    if (COL) {
      const float* A = d.A[cur];
#pragma unroll
      for (int t = 0; t < R; ++t) vec[t] = A[j * R + t];
    } else {
      const float* B = d.B[cur];
#pragma unroll
      for (int t = 0; t < R; ++t) vec[t] = B[(int64_t)t * d.n2 + j];
    }
  }
  float den = 0.f;
  if (live) {
    for (int a = a0; a < a1; ++a) {
      float* cell = tileS + (size_t)a * kPanelCols + c;
      const float dv = *cell;
      const float v = panel_value(dv, lowrank_entry<R>(side + (size_t)a * R, vec), zeta);
      *cell = v;
      den = fmaf(dv, dv, den);
#pragma unroll
      for (int t = 0; t < R; ++t) acc[t] = fmaf(proj[(size_t)a * R + t], v, acc[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) part[((size_t)h * kPanelCols + c) * R + t] = acc[t];
  __syncthreads();
  float out[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    float s = 0.f;
#pragma unroll
    for (int hh = 0; hh < kPanelSplit; ++hh) s += part[((size_t)hh * kPanelCols + c) * R + t];
    out[t] = s;
  }
  float num = 0.f;
  if (live) {
    for (int a = a0; a < a1; ++a) {
      const float v = tileS[(size_t)a * kPanelCols + c];
      float w = 0.f;
#pragma unroll
      for (int t = 0; t < R; ++t) w = fmaf(recon[(size_t)a * R + t], out[t], w);
      const float rr = v - w;
      num = fmaf(rr, rr, num);
    }
    if (h == 0) {
      if (COL) {
        float* An = d.A[nxt];
#pragma unroll
        for (int t = 0; t < R; ++t) An[j * R + t] = out[t];
      } else {
        float* Bn = d.B[nxt];
#pragma unroll
        for (int t = 0; t < R; ++t) Bn[(int64_t)t * d.n2 + j] = out[t];
      }
    }
  }
  acc2[0] += (double)num;
  acc2[1] += (double)den;
}

// Both passes in one grid (row tiles first); the last block to finish reduces
// the per-block partial sums in a fixed order, evaluates e_{k+1}, advances k
// and zeta, and drives the graph's while-node (Alg. 1: "while e_k > epsilon").
template <int R>
__global__ void __launch_bounds__(kPanelThreads) pass_kernel(IterDesc d) {
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
  double acc[2] = {0.0, 0.0};
  if ((int)blockIdx.x < d.nRowTiles)
    panel_pass<R, false>(d, blockIdx.x, k, zeta, smem, acc);
  else
    panel_pass<R, true>(d, blockIdx.x - d.nRowTiles, k, zeta, smem, acc);

  __shared__ double red[4][kPanelThreads / 32];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double v = warp_sum(acc[q]);
    if (lane == 0) red[q][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < kPanelThreads / 32; ++w) s += red[threadIdx.x][w];
    d.partials[(size_t)blockIdx.x * 2 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // warp q: q = 0,1 row-pass num/den; q = 2,3 column-pass num/den
  if (warp < 4) {
    const int colside = warp >> 1, which = warp & 1;
    const unsigned b0 = colside ? (unsigned)d.nRowTiles : 0u;
    const unsigned b1 = colside ? gridDim.x : (unsigned)d.nRowTiles;
    double s = 0.0;
    const volatile double* pv = d.partials;
    for (unsigned b = b0 + lane; b < b1; b += 32) s += pv[(size_t)b * 2 + which];
    s = warp_sum(s);
    if (lane == 0) red[2 + (warp >> 1)][warp & 1] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double num = sqrt(red[2][0]) + sqrt(red[3][0]);
    const double den = sqrt(red[2][1]) + sqrt(red[3][1]);
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

size_t pass_smem_bytes(int nI, int nJ, int Rpad) {
  const int m = nI > nJ ? nI : nJ;
  return (size_t)m * kPanelCols * 4 + 3 * (size_t)m * Rpad * 4 + (size_t)kPanelSplit * kPanelCols * Rpad * 4 +
         8 + 16;
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
  const size_t bytes = pass_smem_bytes(d.nI, d.nJ, R);
  cudaError_t e = cudaFuncSetAttribute(pass_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  pass_kernel<R><<<d.nRowTiles + d.nColTiles, kPanelThreads, bytes, s>>>(d);
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
