// Rank-r truncation H_r of the |I| x |J| core and its pseudo-inverse
// (Alg. 1 Phase II; Sec. 3.1: U_{k+1} = H_r([D - S_{k+1}]_{I,J}),
// U^+ = V_r Sigma_r^{-1} W_r^T).
//
// One CTA of 512 threads.  The dominant rank-r singular subspaces are found
// by two-sided subspace (orthogonal) iteration with Cholesky QR, warm-started
// from the previous iterate's right factor B_k(:,J)^T, whose row space is the
// right singular subspace of L_k(I,J); the core of iteration k+1 differs from
// L_k(I,J) only where the threshold decisions differ.  One step is
//     P = core X,  Y Rp = P (CholQR),  Q = core^T Y,
// and the iteration stops once E = Q - X Rp^T, the part of core^T Y outside
// span X, is below 1e-6 ||Rp||_F (or has stopped shrinking below 1e-5).
// Then Y and X get a second CholQR pass and the r x r Rayleigh-Ritz matrix
// T = Y^T core X follows from the triangular factors without another product
// (T is upper triangular).  With span Y = span W_r and span X = span V_r,
// H_r(core) = Y T X^T and its pseudo-inverse is X T^{-1} Y^T = V_r
// Sigma_r^{-1} W_r^T, so the panel passes need only Y, X T^{-1} and X T^T: no
// r x r SVD on the iteration's path (sigma_kernel computes the singular
// values of T on request).  Pivots of T <= max(|I|,|J|) * FLT_EPSILON times
// the largest are dropped (numerical rank, IRCUR_FLAG_WRANK).
//
// Layout: the core sits in shared memory (one bulk copy) with a leading
// dimension ldu = 4 (mod 8) floats, so 16-byte row vectors read by lanes on
// consecutive rows hit distinct banks.  The m x r blocks X, Y, Q and the
// partial sums are column-major (entry (i, t) at t * ldm + i): lanes always
// run over i, so every access is conflict-free or a broadcast.
//
// Precision: FP32 throughout.  GB300's FP64 pipe runs at a small fraction of
// its FP32 rate, and serial FP64 Cholesky/sqrt/divide chains cost more than
// the whole rest of the iteration; CholQR2 (the second pass) restores
// orthogonality to FP32 rounding.
#include <float.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"
#include "sampler.cuh"

namespace ircur {

template <int R>
struct SvdThreads {
  static constexpr int value = 512;
};
constexpr int kProdChunks = 8;  // max inner-dimension chunks of a core product
constexpr int kSmallMats = 9;   // G, Rp, U, U2y, U2x, T, Ut, Vt, scratch (R x R each)
constexpr size_t kSvdSmemBudget = 220 * 1024;

__host__ __device__ constexpr int round_up4(int x) { return (x + 3) & ~3; }

struct SvdLayout {
  int ldu;  // leading dimension of the core (== ldCore: multiple of 4, ldu/4 odd)
  int ldm;  // column stride of the m x R blocks: max(nI, nJ) rounded up to 4
  int pch;  // inner-dimension chunks the partial-sum buffer holds (1..kProdChunks)
  size_t off_us, off_x, off_y, off_q, off_part, off_small, off_bar, total;
};

__host__ __device__ inline SvdLayout svd_layout(int nI, int nJ, int ldCore, int R, bool core_in_smem) {
  SvdLayout L;
  L.ldu = ldCore;
  L.ldm = round_up4(nI > nJ ? nI : nJ);
  const size_t blk = (size_t)L.ldm * R * 4;
  const size_t small = (size_t)kSmallMats * R * R * 4 + 4 * 32 * 4 + 64;
  const size_t fixed = (core_in_smem ? (size_t)nI * L.ldu * 4 : 0) + 3 * blk + small + 16;
  int pch = fixed < kSvdSmemBudget ? (int)((kSvdSmemBudget - fixed) / blk) : 0;
  L.pch = pch < 1 ? 1 : (pch > kProdChunks ? kProdChunks : pch);
  size_t off = 0;
  L.off_us = off;
  if (core_in_smem) off += (size_t)nI * L.ldu * 4;
  L.off_x = off;
  off += blk;
  L.off_y = off;
  off += blk;
  L.off_q = off;
  off += blk;
  L.off_part = off;
  off += (size_t)L.pch * blk;
  L.off_small = off;
  off += small;
  off = (off + 7) & ~(size_t)7;
  L.off_bar = off;
  off += 8;
  L.total = (off + 15) & ~(size_t)15;
  return L;
}

static int ld_core(int nJ) {
  int ld = (nJ + 3) & ~3;
  if (((ld / 4) & 1) == 0) ld += 4;
  return ld;
}

// The core stays in shared memory when that leaves room for at least two
// partial-sum chunks; otherwise the products read it from global memory (L2).
size_t svd_smem_bytes(int nI, int nJ, int Rpad, bool* core_in_smem) {
  const int ldc = ld_core(nJ);
  SvdLayout L = svd_layout(nI, nJ, ldc, Rpad, true);
  size_t bytes;
  if (L.pch >= 2 && L.total <= kSvdSmemBudget) {
    *core_in_smem = true;
    bytes = L.total;
  } else {
    *core_in_smem = false;
    bytes = svd_layout(nI, nJ, ldc, Rpad, false).total;
  }
  return bytes > sizeof(SamplerSmem) ? bytes : sizeof(SamplerSmem);  // the sampler blocks share the launch
}

struct SvdSmall {
  float* G;     // R x R Gram matrix
  float* Rp;    // R x R factor of the last P = core X
  float* U;     // R x R upper Cholesky factor of the last cholqr
  float* U2y;   // second-pass factor of Y
  float* U2x;   // second-pass factor of X
  float* T;     // R x R Rayleigh-Ritz matrix
  float* Ut;    // R x R
  float* Vt;    // R x R
  float* tmp;   // R x R
  float* dinv;  // R reciprocal pivots
  float* sig;   // R
  float* red;   // 64 reduction slots
  int* ibuf;    // 16 ints
};

// Adds the partial sums of a product (chunk-major, column-major blocks) in a
// fixed order; every (column, row) output is one thread's sum.
template <int R>
__device__ __forceinline__ void reduce_parts(const float* part, int nch, int nout, int ldm, float* out) {
  __syncthreads();
  for (int q = threadIdx.x; q < R * nout; q += blockDim.x) {
    const int t = q / nout, o = q - t * nout;
    const float* pp = part + (size_t)t * ldm + o;
    float s = 0.f;
    for (int c = 0; c < nch; ++c) s += pp[(size_t)c * R * ldm];
    out[(size_t)t * ldm + o] = s;
  }
  __syncthreads();
}

// out = core X (nout = |I| rows, inner nin = |J|).  A thread owns RB rows
// spaced G apart (lanes on consecutive rows) and an inner chunk; core rows are
// read as 16-byte vectors and each 4-row slab of every column of X is a
// 16-byte broadcast shared by the RB rows.  Rows of X beyond nin are zero.
template <int R, int RB = 2>
__device__ void core_times(const float* __restrict__ U, int ldu, int nout, int nin, const float* __restrict__ in,
                           float* __restrict__ out, float* part, int ldm, int pch) {
  const int G = (nout + RB - 1) / RB;
  const int lanes = (G + 31) & ~31;
  int nch = (int)blockDim.x / lanes;
  nch = nch < 1 ? 1 : (nch > pch ? pch : nch);
  const int c = threadIdx.x / lanes, og = threadIdx.x % lanes;
  const int nin4 = round_up4(nin);
  const int qc = round_up4((nin4 + nch - 1) / nch);
  if (c < nch && og < G) {
    float acc[RB][R];
#pragma unroll
    for (int kk = 0; kk < RB; ++kk)
#pragma unroll
      for (int t = 0; t < R; ++t) acc[kk][t] = 0.f;
    const int q0 = c * qc, q1 = q0 + qc < nin4 ? q0 + qc : nin4;
    for (int q = q0; q < q1; q += 4) {
      float4 u[RB];
#pragma unroll
      for (int kk = 0; kk < RB; ++kk) {
        const int o = og + kk * G;
        u[kk] = o < nout ? *reinterpret_cast<const float4*>(U + (size_t)o * ldu + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const float4 x = *reinterpret_cast<const float4*>(in + (size_t)t * ldm + q);
#pragma unroll
        for (int kk = 0; kk < RB; ++kk) {
          float a = acc[kk][t];
          a = fmaf(u[kk].x, x.x, a);
          a = fmaf(u[kk].y, x.y, a);
          a = fmaf(u[kk].z, x.z, a);
          a = fmaf(u[kk].w, x.w, a);
          acc[kk][t] = a;
        }
      }
    }
#pragma unroll
    for (int kk = 0; kk < RB; ++kk) {
      const int o = og + kk * G;
      if (o < nout) {
#pragma unroll
        for (int t = 0; t < R; ++t) part[(size_t)c * R * ldm + (size_t)t * ldm + o] = acc[kk][t];
      }
    }
  }
  reduce_parts<R>(part, nch, nout, ldm, out);
}

// out = core^T Y (nout = |J| rows, inner nin = |I|).  A thread owns four
// consecutive output rows j..j+3 (a 16-byte vector of every core row; lanes on
// consecutive vectors) and an inner chunk stepped by 4: four core vectors and
// one 16-byte broadcast of four rows of Y per column, 16 R FMAs.  Rows of Y
// beyond nin are zero, columns of the core beyond nout are zero.
template <int R>
__device__ void core_t_times(const float* __restrict__ U, int ldu, int nout, int nin, const float* __restrict__ in,
                             float* __restrict__ out, float* part, int ldm, int pch) {
  const int G = (nout + 3) / 4;  // column groups
  const int lanes = (G + 31) & ~31;
  int nch = (int)blockDim.x / lanes;
  nch = nch < 1 ? 1 : (nch > pch ? pch : nch);
  const int c = threadIdx.x / lanes, g = threadIdx.x % lanes;
  const int nin4 = round_up4(nin);
  const int ic = round_up4((nin4 + nch - 1) / nch);
  if (c < nch && g < G) {
    const int j = 4 * g;
    float acc[4][R];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int t = 0; t < R; ++t) acc[e][t] = 0.f;
    const int i0 = c * ic, i1 = i0 + ic < nin4 ? i0 + ic : nin4;
    for (int i = i0; i < i1; i += 4) {
      float4 u[4];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        u[kk] = (i + kk < nin) ? *reinterpret_cast<const float4*>(U + (size_t)(i + kk) * ldu + j)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const float4 y = *reinterpret_cast<const float4*>(in + (size_t)t * ldm + i);
        acc[0][t] = fmaf(u[3].x, y.w, fmaf(u[2].x, y.z, fmaf(u[1].x, y.y, fmaf(u[0].x, y.x, acc[0][t]))));
        acc[1][t] = fmaf(u[3].y, y.w, fmaf(u[2].y, y.z, fmaf(u[1].y, y.y, fmaf(u[0].y, y.x, acc[1][t]))));
        acc[2][t] = fmaf(u[3].z, y.w, fmaf(u[2].z, y.z, fmaf(u[1].z, y.y, fmaf(u[0].z, y.x, acc[2][t]))));
        acc[3][t] = fmaf(u[3].w, y.w, fmaf(u[2].w, y.z, fmaf(u[1].w, y.y, fmaf(u[0].w, y.x, acc[3][t]))));
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (j + e < nout) {
#pragma unroll
        for (int t = 0; t < R; ++t) part[(size_t)c * R * ldm + (size_t)t * ldm + j + e] = acc[e][t];
      }
    }
  }
  reduce_parts<R>(part, nch, nout, ldm, out);
}

template <int R>
__device__ __forceinline__ float sel(const float (&g)[R], int t) {
  float v = 0.f;
#pragma unroll
  for (int u = 0; u < R; ++u)
    if (u == t) v = g[u];
  return v;
}

// Cholesky QR of the nrows x r block Min (column-major, stride ldm) into Mout
// (may alias): Min = Mout U with U upper triangular (written to Uout).  The
// Gram matrix is formed by warps (one entry per warp), factorised by warp 0
// (lane l holds row l of the Schur complement), and applied by forward
// substitution row by row.  Pivots <= 1e-12 of the largest diagonal entry
// mark dependent columns: they become zero columns and are counted.
template <int R>
__device__ int cholqr(const float* Min, float* Mout, int nrows, int r, int ldm, float* Uout, const SvdSmall& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int npairs = r * (r + 1) / 2;
  for (int p = warp; p < npairs; p += nwarps) {
    int s = 0, rem = p;
    while (rem >= r - s) {
      rem -= r - s;
      ++s;
    }
    const int t = s + rem;
    const float* ms = Min + (size_t)s * ldm;
    const float* mt = Min + (size_t)t * ldm;
    float acc = 0.f;
    for (int i = lane; i < nrows; i += 32) acc = fmaf(ms[i], mt[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) {
      sm.G[s * R + t] = acc;
      sm.G[t * R + s] = acc;
    }
  }
  __syncthreads();
  if (warp == 0) {
    float g[R];
#pragma unroll
    for (int u = 0; u < R; ++u) g[u] = (lane < r && u < r) ? sm.G[lane * R + u] : 0.f;
    float maxd = sel<R>(g, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxd = fmaxf(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
    int brk = 0;
    for (int t = 0; t < r; ++t) {
      const float gt = sel<R>(g, t);  // entry (lane, t) = (t, lane) of the Schur complement
      const float dgt = __shfl_sync(0xffffffffu, gt, t);
      const bool keep = dgt > 1e-12f * maxd && dgt <= FLT_MAX;
      const float rinv = keep ? rsqrtf(dgt) : 0.f;
      const float ul = gt * rinv;  // U(t, lane)
      float urow[R];
#pragma unroll
      for (int u = 0; u < R; ++u) urow[u] = __shfl_sync(0xffffffffu, ul, u);  // U(t, u)
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < R; ++u) Uout[t * R + u] = (u >= t) ? urow[u] : 0.f;
        sm.dinv[t] = rinv;
      }
      if (lane > t) {
#pragma unroll
        for (int u = 0; u < R; ++u) g[u] = fmaf(-ul, urow[u], g[u]);
      }
      brk += keep ? 0 : 1;
    }
    if (lane == 0) {
      for (int t = r; t < R; ++t) {
        sm.dinv[t] = 0.f;
        for (int u = 0; u < R; ++u) Uout[t * R + u] = 0.f;
      }
      sm.ibuf[0] = brk;
    }
  }
  __syncthreads();
  // Mout = Min U^{-1}: forward substitution y U = m for every row
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    float m[R], y[R];
#pragma unroll
    for (int s = 0; s < R; ++s) m[s] = Min[(size_t)s * ldm + i];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float v = m[t];
#pragma unroll
      for (int s = 0; s < t; ++s) v = fmaf(-y[s], Uout[s * R + t], v);
      y[t] = v * sm.dinv[t];
    }
#pragma unroll
    for (int t = 0; t < R; ++t) Mout[(size_t)t * ldm + i] = y[t];
  }
  const int brk = sm.ibuf[0];
  __syncthreads();
  return brk;
}

__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t ctr) {
  const uint64_t h = splitmix64(seed ^ splitmix64(ctr));
  return (float)(h >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f;
}

// Round-robin (circle method) partner of player p in round k of n (even) players.
__device__ __forceinline__ int rr_partner(int p, int k, int n) {
  if (p == n - 1) return k;
  if (p == k) return n - 1;
  int q = (2 * k - p) % (n - 1);
  return q < 0 ? q + n - 1 : q;
}

// CS: the core is held in shared memory (a compile-time property, so that
// every core access compiles to a shared-memory load).
template <int R, bool CS>
__device__ __forceinline__ void svd_body(const IterDesc& d, int role, unsigned char* smem) {
  constexpr bool core_in_smem = CS;
  State* st = d.st;
  if (st->done || st->status) return;
  const int k = st->k;
  if (role > 0) {
    // IRCUR-R drawing its own index sets: blocks 1 and 2 draw I_{k+1}, J_{k+1}
    // on otherwise idle SMs while block 0 factorises the core (nothing in this
    // iteration reads them; the next iteration's core kernel does)
    const int axis = role - 1;
    if (d.sampleAhead && k + 1 < d.max_iter) {
      int* out = axis ? const_cast<int*>(d.J_all) + (int64_t)(k + 1) * d.nJ
                      : const_cast<int*>(d.I_all) + (int64_t)(k + 1) * d.nI;
      sample_subset(d.seed, k + 1, axis, axis ? d.n2 : d.n1, axis ? d.nJ : d.nI, out,
                    *reinterpret_cast<SamplerSmem*>(smem));
    }
    return;
  }
  trace_start(d.trace, 3 * k + 1);
  const int nI = d.nI, nJ = d.nJ, r = d.r;
  const SvdLayout L = svd_layout(nI, nJ, d.ldCore, R, core_in_smem);
  const int ldm = L.ldm, ldu = L.ldu;
  float* Us = core_in_smem ? reinterpret_cast<float*>(smem + L.off_us) : d.core;
  float* X = reinterpret_cast<float*>(smem + L.off_x);
  float* Y = reinterpret_cast<float*>(smem + L.off_y);
  float* Q = reinterpret_cast<float*>(smem + L.off_q);
  float* part = reinterpret_cast<float*>(smem + L.off_part);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  SvdSmall sm;
  {
    float* p = reinterpret_cast<float*>(smem + L.off_small);
    sm.G = p;
    p += R * R;
    sm.Rp = p;
    p += R * R;
    sm.U = p;
    p += R * R;
    sm.U2y = p;
    p += R * R;
    sm.U2x = p;
    p += R * R;
    sm.T = p;
    p += R * R;
    sm.Ut = p;
    p += R * R;
    sm.Vt = p;
    p += R * R;
    sm.tmp = p;
    p += R * R;
    sm.dinv = p;
    p += 32;
    sm.sig = p;
    p += 32;
    sm.red = p;
    p += 64;
    sm.ibuf = reinterpret_cast<int*>(p);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  // ---- core into shared memory: one bulk copy (TMA engine) of nI x ldu floats
  const unsigned core_bytes = (unsigned)((size_t)nI * ldu * 4);
  if (core_in_smem && threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, core_bytes);
    bulk_g2s(Us, d.core, core_bytes, bar);
  }
  // ---- X, Y, Q zeroed (padding rows must read as zero); warm start X = B_k(:,J)^T
  for (int q = threadIdx.x; q < 3 * R * ldm; q += blockDim.x) X[q] = 0.f;  // X, Y, Q are contiguous
  __syncthreads();
  for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
#pragma unroll
    for (int t = 0; t < R; ++t) X[(size_t)t * ldm + b] = (t < r) ? d.BJt[(size_t)b * R + t] : 0.f;
  }
  __syncthreads();
  int brk = cholqr<R>(X, X, nJ, r, ldm, sm.U, sm);
  if (brk > 0) {  // first iteration (B_0 = 0) or a deficient factor: random start
    for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
#pragma unroll
      for (int t = 0; t < R; ++t)
        X[(size_t)t * ldm + b] =
            (t < r) ? hash_uniform(d.seed ^ 0x5bd1e995ull, ((uint64_t)k << 32) ^ (uint64_t)(b * R + t)) : 0.f;
    }
    __syncthreads();
    cholqr<R>(X, X, nJ, r, ldm, sm.U, sm);
  }
  if (core_in_smem) {
    bool ok = mbar_wait_bounded(bar, 0, d.spinLimit);
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(&st->status, (int)IRCUR_ETIMEOUT);
      mbar_wait_bounded(bar, 0, kSpinLimit);  // let the copy land before the block exits
    }
    if (!__syncthreads_and(ok)) return;
  }

  // ---- subspace iteration
  int steps = 0;
  bool converged = false;
  float prev_res = 0.f;
  while (true) {
    ++steps;
    core_times<R>(Us, ldu, nI, nJ, X, Y, part, ldm, L.pch);    // Y = core X
    cholqr<R>(Y, Y, nI, r, ldm, sm.Rp, sm);                    // Y Rp = core X
    core_t_times<R>(Us, ldu, nJ, nI, Y, Q, part, ldm, L.pch);  // Q = core^T Y
    // ||Q - X Rp^T||_F^2 and ||Rp||_F^2 in one block reduction
    float e2 = 0.f;
    for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
      float xr[R];
#pragma unroll
      for (int t = 0; t < R; ++t) xr[t] = X[(size_t)t * ldm + b];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = Q[(size_t)t * ldm + b];
#pragma unroll
        for (int s2 = t; s2 < R; ++s2) v = fmaf(-xr[s2], sm.Rp[t * R + s2], v);
        e2 = fmaf(v, v, e2);
      }
    }
    float rc2 = 0.f;
    if (threadIdx.x < R * R) rc2 = sm.Rp[threadIdx.x] * sm.Rp[threadIdx.x];
    e2 = warp_sum(e2);
    rc2 = warp_sum(rc2);
    if (lane == 0) {
      sm.red[warp] = e2;
      sm.red[32 + warp] = rc2;
    }
    __syncthreads();
    float E2 = 0.f, RC2 = 0.f;
    for (int w = 0; w < nwarps; ++w) {
      E2 += sm.red[w];
      RC2 += sm.red[32 + w];
    }
    const float res = sqrtf(E2), nrm = sqrtf(RC2);
    if (res <= 1e-6f * nrm || (steps > 1 && res > 0.5f * prev_res && res <= 1e-5f * nrm) || !(nrm > 0.f)) {
      converged = true;
      break;
    }
    if (steps >= d.svdMaxSteps) break;  // keep X, Y, Rp of the same step
    prev_res = res;
    cholqr<R>(Q, X, nJ, r, ldm, sm.U, sm);  // X = orth(core^T Y)
  }

  // ---- second CholQR passes; T = U2y Rp U2x^{-1} = Y^T core X for the new bases
  cholqr<R>(Y, Y, nI, r, ldm, sm.U2y, sm);
  cholqr<R>(X, X, nJ, r, ldm, sm.U2x, sm);
  if (threadIdx.x < 32) {
    const int s = threadIdx.x;
    if (s < r) {
      float row[R];  // (U2y Rp)(s, :)
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = 0.f;
        for (int u = 0; u < r; ++u) v = fmaf(sm.U2y[s * R + u], sm.Rp[u * R + t], v);
        row[t] = v;
      }
      // T(s,:) U2x = row  (forward substitution; dropped pivots give zeros)
      float tr[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = row[t];
#pragma unroll
        for (int u = 0; u < t; ++u) v = fmaf(-tr[u], sm.U2x[u * R + t], v);
        tr[t] = (t < r) ? v * sm.dinv[t] : 0.f;
      }
#pragma unroll
      for (int t = 0; t < R; ++t) sm.T[s * R + t] = tr[t];
    }
  }
  __syncthreads();

  // ---- numerical rank from the diagonal of the upper-triangular T (its
  // singular values up to the off-diagonal part, which the iteration has
  // driven below 1e-6 of ||T||), and the inverse of T on the kept pivots.
  if (warp == 0) {
    const float dabs = lane < r ? fabsf(sm.T[lane * R + lane]) : 0.f;
    float dmax = dabs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    const float tol = (float)(nI > nJ ? nI : nJ) * FLT_EPSILON * dmax;
    const bool keep = lane < r && dabs > tol && dabs > 0.f;
    const unsigned kmask = __ballot_sync(0xffffffffu, keep);
    if (lane < r) {  // column `lane` of T^{-1} by back substitution, in registers
      const int c = lane;
      float x[R];
#pragma unroll
      for (int s2 = R - 1; s2 >= 0; --s2) {
        float v = 0.f;
        if (s2 <= c && ((kmask >> s2) & 1u)) {
          v = (s2 == c) ? 1.f : 0.f;
#pragma unroll
          for (int u = s2 + 1; u < R; ++u)
            if (u <= c) v = fmaf(-sm.T[s2 * R + u], x[u], v);
          v = v / sm.T[s2 * R + s2];
        }
        x[s2] = v;
      }
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) sm.tmp[s2 * R + c] = x[s2];
      sm.sig[lane] = keep ? dabs : 0.f;
    }
    if (lane == 0) {
      sm.ibuf[1] = __popc(kmask);
      sm.ibuf[2] = (int)kmask;
      for (int t = r; t < R; ++t) {
        sm.sig[t] = 0.f;
        for (int u = 0; u < R; ++u) sm.tmp[u * R + t] = 0.f;
      }
    }
  }
  __syncthreads();
  const int rank = sm.ibuf[1];
  const unsigned kmask = (unsigned)sm.ibuf[2];
  // Outputs for the panel passes (U^+ = X T^{-1} Y^T, the pseudo-inverse of
  // H_r(core) = Y T X^T):
  //   W  = Y          (row pass: B_{k+1} = Y^T R, residual R - Y Y^T R),
  //   Vs = X T^{-1}   (column pass: A_{k+1} = C X T^{-1}),
  //   V  = X T^T      (column pass residual C - A_{k+1} T X^T = C - C X X^T).
  for (int i = threadIdx.x; i < nI; i += blockDim.x) {
#pragma unroll
    for (int t = 0; t < R; ++t) d.W[(size_t)i * R + t] = ((kmask >> t) & 1u) ? Y[(size_t)t * ldm + i] : 0.f;
  }
  for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
    float x[R];
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) x[s2] = X[(size_t)s2 * ldm + b];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float vp = 0.f, vr = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) {
        vp = fmaf(x[s2], sm.tmp[s2 * R + t], vp);
        vr = fmaf(x[s2], sm.T[t * R + s2], vr);
      }
      const bool kt = (kmask >> t) & 1u;
      d.Vs[(size_t)b * R + t] = kt ? vp : 0.f;
      d.V[(size_t)b * R + t] = kt ? vr : 0.f;
    }
  }
  if (threadIdx.x < R) d.sigma[threadIdx.x] = sm.sig[threadIdx.x];
  if (threadIdx.x < R * R) d.Tm[threadIdx.x] = sm.T[threadIdx.x];
  if (threadIdx.x == 0) {
    unsigned f = 0u;
    if (rank < r) f |= IRCUR_FLAG_WRANK;
    if (!converged) f |= IRCUR_FLAG_SVD_NOCONV;
    if (f) atomicOr(&st->flags, f);
    st->svd_steps += steps;
    st->svd_last_steps = steps;
  }
  if (d.trace) {
    __syncthreads();
    trace_stop(d.trace, 3 * d.max_iter, 3 * k + 1);
  }
}

template <int R, bool CS>
__global__ void __launch_bounds__(SvdThreads<R>::value, 1) svd_kernel(IterDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  svd_body<R, CS>(d, blockIdx.x, smem);
}

// Batched form: blockIdx.x indexes `list` (the instances of one core-layout
// group), blockIdx.y is the role (0: core SVD, 1 and 2: next index sets).
template <int R, bool CS>
__global__ void __launch_bounds__(SvdThreads<R>::value, 1) svd_batch_kernel(const IterDesc* __restrict__ ds,
                                                                           const int* __restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  svd_body<R, CS>(ds[list[blockIdx.x]], blockIdx.y, smem);
}

// Singular values of the last Rayleigh-Ritz matrix T (the r largest singular
// values of the last core, descending): one-sided Jacobi in one warp, lane p
// owning column p, round-robin pair ordering.  Used on request only.
template <int R>
__global__ void sigma_kernel(const float* __restrict__ Tm, int r, float* __restrict__ sigma) {
  const int p = threadIdx.x;
  float tc[R];
#pragma unroll
  for (int i = 0; i < R; ++i) tc[i] = (p < r && i < r) ? Tm[i * R + p] : 0.f;
  const int nplay = (r + 1) & ~1;
  for (int sweep = 0; sweep < 30; ++sweep) {
    int rotated = 0;
    for (int rnd = 0; rnd < nplay - 1; ++rnd) {
      const int q = (p < nplay) ? rr_partner(p, rnd, nplay) : p;
      float tq[R];
#pragma unroll
      for (int i = 0; i < R; ++i) tq[i] = __shfl_sync(0xffffffffu, tc[i], q);
      if (p < r && q < r && q != p) {
        const bool lo = p < q;
        float app = 0.f, aqq = 0.f, apq = 0.f;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const float a = lo ? tc[i] : tq[i];
          const float b = lo ? tq[i] : tc[i];
          app = fmaf(a, a, app);
          aqq = fmaf(b, b, aqq);
          apq = fmaf(a, b, apq);
        }
        if (fabsf(apq) > 1e-6f * sqrtf(app * aqq)) {
          rotated = 1;
          const float zeta = (aqq - app) / (2.f * apq);
          const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = rsqrtf(1.f + tt * tt), s = c * tt;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const float a = lo ? tc[i] : tq[i], b = lo ? tq[i] : tc[i];
            tc[i] = lo ? (c * a - s * b) : (s * a + c * b);
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, rotated)) break;
  }
  float s2 = 0.f;
#pragma unroll
  for (int i = 0; i < R; ++i) s2 = fmaf(tc[i], tc[i], s2);
  const float sg = (p < r) ? sqrtf(s2) : -1.f;
  int pos = 0;
  for (int q = 0; q < r; ++q) {
    const float sq = __shfl_sync(0xffffffffu, sg, q);
    pos += (sq > sg) || (sq == sg && q < p);
  }
  if (p < r) sigma[pos] = sg;
}

template <int R>
static cudaError_t launch_sigma_r(const float* Tm, int r, float* sigma, cudaStream_t s) {
  sigma_kernel<R><<<1, 32, 0, s>>>(Tm, r, sigma);
  return cudaGetLastError();
}

cudaError_t launch_sigma(const float* Tm, int r, int Rpad, float* sigma, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_sigma_r<1>(Tm, r, sigma, s);
    case 2: return launch_sigma_r<2>(Tm, r, sigma, s);
    case 3: return launch_sigma_r<3>(Tm, r, sigma, s);
    case 4: return launch_sigma_r<4>(Tm, r, sigma, s);
    case 5: return launch_sigma_r<5>(Tm, r, sigma, s);
    case 6: return launch_sigma_r<6>(Tm, r, sigma, s);
    case 7: return launch_sigma_r<7>(Tm, r, sigma, s);
    case 8: return launch_sigma_r<8>(Tm, r, sigma, s);
    case 9: return launch_sigma_r<9>(Tm, r, sigma, s);
    case 10: return launch_sigma_r<10>(Tm, r, sigma, s);
    case 12: return launch_sigma_r<12>(Tm, r, sigma, s);
    case 16: return launch_sigma_r<16>(Tm, r, sigma, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int R>
static cudaError_t launch_svd_r(const IterDesc& d, cudaStream_t s) {
  bool in_smem = false;
  const size_t bytes = svd_smem_bytes(d.nI, d.nJ, R, &in_smem);
  if (in_smem) {
    cudaError_t e = cudaFuncSetAttribute(svd_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    svd_kernel<R, true><<<1 + (d.sampleAhead ? 2 : 0), SvdThreads<R>::value, bytes, s>>>(d);
  } else {
    cudaError_t e = cudaFuncSetAttribute(svd_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    svd_kernel<R, false><<<1 + (d.sampleAhead ? 2 : 0), SvdThreads<R>::value, bytes, s>>>(d);
  }
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_svd_batch_r(const BatchLaunch& b, cudaStream_t s) {
  if (b.svd_n[0] > 0) {
    cudaError_t e = cudaFuncSetAttribute(svd_batch_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)b.svd_smem[0]);
    if (e != cudaSuccess) return e;
    svd_batch_kernel<R, true><<<dim3(b.svd_n[0], b.svd_roles), SvdThreads<R>::value, b.svd_smem[0], s>>>(
        b.ds, b.svd_list[0]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (b.svd_n[1] > 0) {
    cudaError_t e = cudaFuncSetAttribute(svd_batch_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)b.svd_smem[1]);
    if (e != cudaSuccess) return e;
    svd_batch_kernel<R, false><<<dim3(b.svd_n[1], b.svd_roles), SvdThreads<R>::value, b.svd_smem[1], s>>>(
        b.ds, b.svd_list[1]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_svd_batch(const BatchLaunch& b, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_svd_batch_r<1>(b, s);
    case 2: return launch_svd_batch_r<2>(b, s);
    case 3: return launch_svd_batch_r<3>(b, s);
    case 4: return launch_svd_batch_r<4>(b, s);
    case 5: return launch_svd_batch_r<5>(b, s);
    case 6: return launch_svd_batch_r<6>(b, s);
    case 7: return launch_svd_batch_r<7>(b, s);
    case 8: return launch_svd_batch_r<8>(b, s);
    case 9: return launch_svd_batch_r<9>(b, s);
    case 10: return launch_svd_batch_r<10>(b, s);
    case 12: return launch_svd_batch_r<12>(b, s);
    case 16: return launch_svd_batch_r<16>(b, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_svd(const IterDesc& d, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_svd_r<1>(d, s);
    case 2: return launch_svd_r<2>(d, s);
    case 3: return launch_svd_r<3>(d, s);
    case 4: return launch_svd_r<4>(d, s);
    case 5: return launch_svd_r<5>(d, s);
    case 6: return launch_svd_r<6>(d, s);
    case 7: return launch_svd_r<7>(d, s);
    case 8: return launch_svd_r<8>(d, s);
    case 9: return launch_svd_r<9>(d, s);
    case 10: return launch_svd_r<10>(d, s);
    case 12: return launch_svd_r<12>(d, s);
    case 16: return launch_svd_r<16>(d, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ircur
