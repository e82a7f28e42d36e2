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
__device__ __forceinline__ void core_body(const IterDesc& d, int blk, int nblk) {
  const State* st = d.st;
  if (st->done || st->status) return;
  const int k = st->k;
  const float zeta = (float)st->zeta;
  const int cur = k & 1;
  const int* I = d.I_all + (d.resample ? (int64_t)k * d.nI : 0);
  const int* J = d.J_all + (d.resample ? (int64_t)k * d.nJ : 0);
  const float* A = d.A[cur];
  const float* B = d.B[cur];
  trace_start(d.trace, 3 * k + 0);
  for (int a = blk; a < d.nI; a += nblk) {
    const int ia = I[a];
    float arow[R];
#pragma unroll
    for (int t = 0; t < R; ++t) arow[t] = A[(int64_t)ia * R + t];
    if (threadIdx.x < R) d.AI[(size_t)a * R + threadIdx.x] = A[(int64_t)ia * R + threadIdx.x];
    const float* rowp = d.rowSrc + (int64_t)(d.resample ? ia : a) * d.rowLd;
    for (int b = threadIdx.x; b < d.nJ; b += blockDim.x) {
      const int j = J[b];
      float bcol[R];
#pragma unroll
      for (int t = 0; t < R; ++t) bcol[t] = B[(int64_t)t * d.n2 + j];
      if (a == 0) {
#pragma unroll
        for (int t = 0; t < R; ++t) d.BJt[(size_t)b * R + t] = bcol[t];
      }
      const float l = lowrank_entry<R>(arow, bcol);
      d.core[(int64_t)a * d.ldCore + b] = panel_value(rowp[j], l, zeta);
    }
  }
  if (d.trace) {
    __syncthreads();
    trace_stop(d.trace, 3 * d.max_iter, 3 * k + 0);
  }
}

template <int R>
__global__ void __launch_bounds__(256) core_kernel(IterDesc d) {
  core_body<R>(d, blockIdx.x, gridDim.x);
}

// Batched form: blockIdx.y selects the instance.
template <int R>
__global__ void __launch_bounds__(256) core_batch_kernel(const IterDesc* __restrict__ ds) {
  core_body<R>(ds[blockIdx.y], blockIdx.x, gridDim.x);
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
// The m x kPanelCols tile is staged in shared memory by 16-byte asynchronous
// copies (the rows are gathered: one small segment per panel row, which the
// per-instruction cost of bulk TMA copies makes slower), overwritten with
// D - S, and read back by the second sweep for the explicit residual.  A
// thread owns two adjacent columns and a contiguous share of the rows
// (kPanelSplit shares); the partial projections are added in a fixed order.
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

  constexpr int RX = (R + 3) & ~3;                         // 16-byte rows of the small matrices
  float* tileS = reinterpret_cast<float*>(smem);           // m x kPanelCols
  float* side = tileS + (size_t)m * kPanelCols;             // m x RX
  float* proj = side + (size_t)m * RX;                      // m x RX
  float* recon = COL ? proj + (size_t)m * RX : proj;        // m x RX (row pass: recon == proj)
  float* part = proj + (size_t)(COL ? 2 : 1) * m * RX;      // kPanelSplit x kPanelCols x RX
  float* outS = part + (size_t)kPanelSplit * kPanelCols * RX;  // kPanelCols x RX

  const int64_t j0 = (int64_t)tile * kPanelCols;
  const int ncols = (int)((ncolsTotal - j0) < kPanelCols ? (ncolsTotal - j0) : kPanelCols);
  const bool vec16 = (COL ? d.colBulk : d.rowBulk) && ncols == kPanelCols;

  // 1. the panel tile: 16-byte asynchronous copies issued first, so that they
  //    fly during the staging of the small matrices
  if (vec16) {
    constexpr int kV = kPanelCols / 4;
    for (int q = threadIdx.x; q < m * kV; q += blockDim.x) {
      const int a = q / kV, c4 = q - a * kV;
      const int64_t row = mapped ? __ldg(map + a) : a;
      cp_async16(tileS + (size_t)a * kPanelCols + 4 * c4, src + row * ld + j0 + 4 * c4);
    }
  } else {
    for (int q = threadIdx.x; q < m * kPanelCols; q += blockDim.x) {
      const int a = q / kPanelCols, c = q - a * kPanelCols;
      const int64_t row = mapped ? map[a] : a;
      tileS[q] = c < ncols ? src[row * ld + j0 + c] : 0.f;
    }
  }
  // 2. the m x R side, projection and reconstruction matrices (rows padded to RX)
  {
    const float* sideG = COL ? d.BJt : d.AI;
    for (int q = threadIdx.x; q < m * RX; q += blockDim.x) {
      const int a = q / RX, t = q - a * RX;
      const bool in = t < R;
      side[q] = in ? sideG[a * R + t] : 0.f;
      if (COL) {
        proj[q] = in ? d.Vs[a * R + t] : 0.f;
        recon[q] = in ? d.V[a * R + t] : 0.f;
      } else {
        proj[q] = in ? d.W[a * R + t] : 0.f;
      }
    }
  }
  if (vec16) cp_async_wait_all();
  __syncthreads();

  // thread = (column pair cp, row split h); columns c0 = 2 cp, c0 + 1
  constexpr int kPairs = kPanelCols / 2;
  const int cp = threadIdx.x % kPairs, h = threadIdx.x / kPairs;
  const int c0 = 2 * cp;
  const int a0 = (int)((long long)h * m / kPanelSplit), a1 = (int)((long long)(h + 1) * m / kPanelSplit);
  const bool live0 = c0 < ncols, live1 = c0 + 1 < ncols;
  const int64_t j = j0 + c0;
  float vec0[R], vec1[R], acc0[R], acc1[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    vec0[t] = vec1[t] = 0.f;
    acc0[t] = acc1[t] = 0.f;
  }
  if (COL) {
    const float* A = d.A[cur];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      if (live0) vec0[t] = A[j * R + t];
      if (live1) vec1[t] = A[(j + 1) * R + t];
    }
  } else {
    const float* B = d.B[cur];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      if (live0) vec0[t] = B[(int64_t)t * d.n2 + j];
      if (live1) vec1[t] = B[(int64_t)t * d.n2 + j + 1];
    }
  }
  const float m0 = live0 ? 1.f : 0.f, m1 = live1 ? 1.f : 0.f;
  float den = 0.f;
  for (int a = a0; a < a1; ++a) {
    float2* cell = reinterpret_cast<float2*>(tileS + (size_t)a * kPanelCols + c0);
    const float2 dv = *cell;
    float sr[R], pr[R];
#pragma unroll
    for (int t4 = 0; t4 < RX / 4; ++t4) {
      const float4 sv = *reinterpret_cast<const float4*>(side + (size_t)a * RX + 4 * t4);
      const float4 pv = *reinterpret_cast<const float4*>(proj + (size_t)a * RX + 4 * t4);
      const float s4[4] = {sv.x, sv.y, sv.z, sv.w}, p4[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * t4 + e < R) {
          sr[4 * t4 + e] = s4[e];
          pr[4 * t4 + e] = p4[e];
        }
    }
    const float v0 = panel_value(dv.x, lowrank_entry<R>(sr, vec0), zeta) * m0;
    const float v1 = panel_value(dv.y, lowrank_entry<R>(sr, vec1), zeta) * m1;
    *cell = make_float2(v0, v1);
    den = fmaf(dv.x, dv.x, den);
    den = fmaf(dv.y, dv.y, den);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      acc0[t] = fmaf(pr[t], v0, acc0[t]);
      acc1[t] = fmaf(pr[t], v1, acc1[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) {
    part[((size_t)h * kPanelCols + c0) * RX + t] = acc0[t];
    part[((size_t)h * kPanelCols + c0 + 1) * RX + t] = acc1[t];
  }
  __syncthreads();
  // projections of every column: the kPanelSplit partial sums in a fixed order
  for (int q = threadIdx.x; q < kPanelCols * R; q += blockDim.x) {
    const int cc = q / R, t = q - cc * R;
    float sum = 0.f;
#pragma unroll
    for (int hh = 0; hh < kPanelSplit; ++hh) sum += part[((size_t)hh * kPanelCols + cc) * RX + t];
    outS[cc * RX + t] = sum;
  }
  __syncthreads();
  float out0[R], out1[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    out0[t] = outS[c0 * RX + t];
    out1[t] = outS[(c0 + 1) * RX + t];
  }
  float num = 0.f;
  for (int a = a0; a < a1; ++a) {
    const float2 v = *reinterpret_cast<const float2*>(tileS + (size_t)a * kPanelCols + c0);
    float rr[R];
#pragma unroll
    for (int t4 = 0; t4 < RX / 4; ++t4) {
      const float4 rv = *reinterpret_cast<const float4*>(recon + (size_t)a * RX + 4 * t4);
      const float r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * t4 + e < R) rr[4 * t4 + e] = r4[e];
    }
    float w0 = 0.f, w1 = 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      w0 = fmaf(rr[t], out0[t], w0);
      w1 = fmaf(rr[t], out1[t], w1);
    }
    const float e0 = (v.x - w0) * m0, e1 = (v.y - w1) * m1;
    num = fmaf(e0, e0, num);
    num = fmaf(e1, e1, num);
  }
  if (h == 0) {
    if (COL) {
      float* An = d.A[nxt];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (live0) An[j * R + t] = out0[t];
        if (live1) An[(j + 1) * R + t] = out1[t];
      }
    } else {
      float* Bn = d.B[nxt];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (live0) Bn[(int64_t)t * d.n2 + j] = out0[t];
        if (live1) Bn[(int64_t)t * d.n2 + j + 1] = out1[t];
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
__device__ __forceinline__ void pass_body(const IterDesc& d, int blk, int nblk, unsigned char* smem) {
  State* st = d.st;
  if (st->done || st->status) {
    if (blk == 0 && threadIdx.x == 0) {
      st->done = 1;
      if (d.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)d.cond, 0u);
    }
    return;
  }
  const int k = st->k;
  const float zeta = (float)st->zeta;
  trace_start(d.trace, 3 * k + 2);
  double acc[2] = {0.0, 0.0};
  const int nPanel = d.nRowTiles + d.nColTiles;
  if (blk < d.nRowTiles) {
    panel_pass<R, false>(d, blk, k, zeta, smem, acc);
  } else if (blk < nPanel) {
    panel_pass<R, true>(d, blk - d.nRowTiles, k, zeta, smem, acc);
  }

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
    d.partials[(size_t)blk * 2 + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  trace_stop(d.trace, 3 * d.max_iter, 3 * k + 2);
  if (threadIdx.x == 0) is_last = (atomicAdd(&st->counter, 1u) == (unsigned)nblk - 1u);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // warp q: q = 0,1 row-pass num/den; q = 2,3 column-pass num/den
  if (warp < 4) {
    const int colside = warp >> 1, which = warp & 1;
    const unsigned b0 = colside ? (unsigned)d.nRowTiles : 0u;
    const unsigned b1 = colside ? (unsigned)nblk : (unsigned)d.nRowTiles;
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
    st->zeta_last = st->zeta;
    st->zeta = st->zeta * d.gamma;
    st->counter = 0u;
    const int done = (e <= d.tol) || (k + 1 >= d.max_iter) || (st->status != 0);
    st->done = done;
    __threadfence();
    trace_stop(d.trace, 3 * d.max_iter, 3 * k + 2);
    if (d.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)d.cond, done ? 0u : 1u);
  }
}

template <int R>
__global__ void __launch_bounds__(kPanelThreads, 3) pass_kernel(IterDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  pass_body<R>(d, blockIdx.x, gridDim.x, smem);
}

// Batched form: the grid holds every instance's tiles back to back;
// tile_base[i] is the first block of instance i (tile_base[count] = grid).
template <int R>
__global__ void __launch_bounds__(kPanelThreads, 3) pass_batch_kernel(const IterDesc* __restrict__ ds,
                                                                      const int* __restrict__ tile_base, int count) {
  extern __shared__ __align__(16) unsigned char smem[];
  int lo = 0, hi = count - 1;  // instance i with tile_base[i] <= blockIdx.x < tile_base[i + 1]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile_base[mid] <= (int)blockIdx.x)
      lo = mid;
    else
      hi = mid - 1;
  }
  pass_body<R>(ds[lo], (int)blockIdx.x - tile_base[lo], tile_base[lo + 1] - tile_base[lo], smem);
}

// Batched loop control: the while-node continues while any instance runs.
__global__ void batch_check_kernel(const IterDesc* __restrict__ ds, int count, unsigned long long cond,
                                   int* any_active) {
  __shared__ int act;
  if (threadIdx.x == 0) act = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const State* st = ds[i].st;
    if (!st->done && !st->status) atomicOr(&act, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *any_active = act;
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, act ? 1u : 0u);
  }
}

size_t pass_smem_bytes(int nI, int nJ, int Rpad) {
  const int m = nI > nJ ? nI : nJ;
  const size_t rx = (size_t)((Rpad + 3) & ~3);
  return (size_t)m * kPanelCols * 4 + 3 * (size_t)m * rx * 4 + (size_t)kPanelSplit * kPanelCols * rx * 4 +
         (size_t)kPanelCols * rx * 4 + 16;
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

template <int R>
static cudaError_t launch_batch_iter_r(const BatchLaunch& b, cudaStream_t s) {
  core_batch_kernel<R><<<dim3(b.core_blocks, b.count), 256, 0, s>>>(b.ds);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_svd_batch(b, R, s);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pass_batch_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.pass_smem);
  if (e != cudaSuccess) return e;
  pass_batch_kernel<R><<<b.total_tiles, kPanelThreads, b.pass_smem, s>>>(b.ds, b.tile_base, b.count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_check_kernel<<<1, 256, 0, s>>>(b.ds, b.count, b.cond, b.any_active);
  return cudaGetLastError();
}

cudaError_t launch_batch_iteration(const BatchLaunch& b, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_batch_iter_r<1>(b, s);
    case 2: return launch_batch_iter_r<2>(b, s);
    case 3: return launch_batch_iter_r<3>(b, s);
    case 4: return launch_batch_iter_r<4>(b, s);
    case 5: return launch_batch_iter_r<5>(b, s);
    case 6: return launch_batch_iter_r<6>(b, s);
    case 7: return launch_batch_iter_r<7>(b, s);
    case 8: return launch_batch_iter_r<8>(b, s);
    case 9: return launch_batch_iter_r<9>(b, s);
    case 10: return launch_batch_iter_r<10>(b, s);
    case 12: return launch_batch_iter_r<12>(b, s);
    case 16: return launch_batch_iter_r<16>(b, s);
    default: return cudaErrorInvalidValue;
  }
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
