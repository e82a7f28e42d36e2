// Rank-r truncation H_r of the |I| x |J| core and its pseudo-inverse
// (Alg. 1 Phase II; Sec. 3.1: U_{k+1} = H_r([D - S_{k+1}]_{I,J}),
// U^+ = V_r Sigma_r^{-1} W_r^T).
//
// The dominant rank-r singular subspaces are found by two-sided subspace
// (orthogonal) iteration with Cholesky QR, warm-started from the previous
// iterate's right factor B_k(:,J)^T, whose row space is the right singular
// subspace of L_k(I,J); the core of iteration k+1 differs from L_k(I,J) only
// where the threshold decisions differ.  One step is
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
// It runs on a cluster of CTAs that share the core by rows (csvd_body).
// Layout: the core rows sit in shared memory (one bulk copy per CTA) with a
// leading dimension ldu = 4 (mod 8) floats, so 16-byte row vectors read by
// lanes on consecutive rows hit distinct banks.  The m x r blocks X, Y, Q and
// the partial sums are column-major (entry (i, t) at t * ld + i): lanes run
// over i, so every access is conflict-free or a broadcast.
//
// Precision: FP32 throughout.  GB300's FP64 pipe runs at a small fraction of
// its FP32 rate, and serial FP64 Cholesky/sqrt/divide chains cost more than
// the whole rest of the iteration; CholQR2 (the second pass) restores
// orthogonality to FP32 rounding.
#include <cooperative_groups.h>
#include <float.h>
#include <string.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"
#include "sampler.cuh"

namespace ircur {

namespace cg = cooperative_groups;

constexpr int kSmallMats = 9;   // G, Rp, U, U2y, U2x, T, Ut, Vt, scratch (R x R each)

__host__ __device__ constexpr int round_up4(int x) { return (x + 3) & ~3; }

static int ld_core(int nJ) {
  int ld = (nJ + 3) & ~3;
  if (((ld / 4) & 1) == 0) ld += 4;
  return ld;
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

template <int R>
__device__ __forceinline__ float sel(const float (&g)[R], int t) {
  float v = 0.f;
#pragma unroll
  for (int u = 0; u < R; ++u)
    if (u == t) v = g[u];
  return v;
}

// Cholesky QR of a column-major block, in three pieces (the cluster SVD
// reduces the Gram matrix across its CTAs between the first two).
//
// gram_block: G(s,t) = M(:,s) . M(:,t) over nrows rows for s <= t < r (one
// entry per warp, lanes over rows), both triangles written.
template <int R>
__device__ void gram_block(const float* M, int nrows, int ld, int r, float* G) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int npairs = r * (r + 1) / 2;
  for (int p = warp; p < npairs; p += nwarps) {
    int s = 0, rem = p;
    while (rem >= r - s) {
      rem -= r - s;
      ++s;
    }
    const int t = s + rem;
    const float* ms = M + (size_t)s * ld;
    const float* mt = M + (size_t)t * ld;
    float acc = 0.f;
    for (int i = lane; i < nrows; i += 32) acc = fmaf(ms[i], mt[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) {
      G[s * R + t] = acc;
      G[t * R + s] = acc;
    }
  }
  __syncthreads();
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


// Every warp factorises the same R x R Gram matrix G = U^T U in registers (lane
// l holds row l of the Schur complement) and keeps U and the reciprocal
// pivots in its own shared slot (Uw, dinvw), so the rows it then transforms
// need no block barrier; identical arithmetic gives identical factors in every
// warp and CTA.  Pivots <= 1e-12 of the largest diagonal entry mark dependent
// columns (zero rows of U, dinv = 0).  Returns the number of those.
template <int R>
__device__ int warp_chol(const float* G, int r, float* Uw, float* dinvw) {
  const int lane = threadIdx.x & 31;
  float g[R];
#pragma unroll
  for (int u = 0; u < R; ++u) g[u] = (lane < r && u < r) ? G[lane * R + u] : 0.f;
  float maxd = sel<R>(g, lane);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxd = fmaxf(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
  int brk = 0;
  for (int t = 0; t < r; ++t) {
    const float gt = sel<R>(g, t);
    const float dgt = __shfl_sync(0xffffffffu, gt, t);
    const bool keep = dgt > 1e-12f * maxd && dgt <= FLT_MAX;
    const float rinv = keep ? rsqrtf(dgt) : 0.f;
    const float ul = gt * rinv;  // U(t, lane)
    float urow[R];
#pragma unroll
    for (int u = 0; u < R; ++u) urow[u] = __shfl_sync(0xffffffffu, ul, u);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < R; ++u) Uw[t * R + u] = (u >= t) ? urow[u] : 0.f;
      dinvw[t] = rinv;
    }
    if (lane > t) {
#pragma unroll
      for (int u = 0; u < R; ++u) g[u] = fmaf(-ul, urow[u], g[u]);
    }
    brk += keep ? 0 : 1;
  }
  if (lane == 0) {
    for (int t = r; t < R; ++t) {
      dinvw[t] = 0.f;
      for (int u = 0; u < R; ++u) Uw[t * R + u] = 0.f;
    }
  }
  __syncwarp();
  return brk;
}

// y U = m for one row (forward substitution with U from warp_chol).
template <int R>
__device__ __forceinline__ void row_subst(const float (&m)[R], float (&y)[R], const float* Uw, const float* dinvw) {
#pragma unroll
  for (int t = 0; t < R; ++t) {
    float v = m[t];
#pragma unroll
    for (int s2 = 0; s2 < t; ++s2) v = fmaf(-y[s2], Uw[s2 * R + t], v);
    y[t] = v * dinvw[t];
  }
}

// Cholesky QR of a column-major block (Min -> Mout, may alias) with the factor
// formed by every warp; warp 0's copy goes to Uout / sm.dinv for later use.
template <int R>
__device__ int cholqr_w(const float* Min, int ldin, float* Mout, int ldout, int nrows, int r, float* Uout,
                        const SvdSmall& sm, float* slots) {
  gram_block<R>(Min, nrows, ldin, r, sm.G);
  const int warp = threadIdx.x >> 5;
  float* Uw = warp == 0 ? Uout : slots + (size_t)warp * (R * R + R);
  float* dw = warp == 0 ? sm.dinv : Uw + R * R;
  const int brk = warp_chol<R>(sm.G, r, Uw, dw);
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    float m[R], y[R];
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) m[s2] = Min[(size_t)s2 * ldin + i];
    row_subst<R>(m, y, Uw, dw);
#pragma unroll
    for (int t = 0; t < R; ++t) Mout[(size_t)t * ldout + i] = y[t];
  }
  __syncthreads();
  return brk;
}

// ---------------------------------------------------------------------------
// Core SVD on a thread-block cluster of kSvdCluster CTAs (distributed shared
// memory).  The two-sided subspace iteration above, with the core split by
// rows: CTA c holds rows [c mr, (c+1) mr) of the core in its shared
// memory (one bulk copy), its own rows of Y and a full copy of X:
//   Y_c = core_c X                 local rows, no exchange
//   Gram(Y) = sum_c Y_c^T Y_c      R x R partials summed over the cluster
//   Q = sum_c core_c^T Y_c         full-size partials summed over the cluster
//                                  (every CTA forms the whole sum)
//   Rp, residual, X = orth(Q)      replicated in every CTA
// Every cluster-wide sum adds the CTAs' partials in rank order, so each CTA
// holds bit-identical matrices and takes identical branch decisions; one
// cluster barrier per step (the partial buffers alternate).  Outputs: W by rows of Y (each CTA its rows),
// X T^{-1} and X T^T by slices of rows.
constexpr int kCsvdThreads = 256;

struct CsvdLayout {
  int mr;       // core rows per CTA
  int ldy;      // column stride of the local Y block (mr rounded up to 4)
  int ldx;      // column stride of X and of the Q partial (nJ rounded up to 4)
  int js;       // rows of the outputs X T^{-1}, X T^T each CTA writes
  size_t off_uc, off_x, off_y, off_qp, off_qs, off_qp2, off_end_zero, off_ra, off_ra2, off_stage, off_slots, off_small,
      off_flag,
      off_bar, total;
};

__host__ __device__ inline CsvdLayout csvd_layout(int nI, int nJ, int ldu, int R, int cl) {
  CsvdLayout L;
  L.mr = (nI + cl - 1) / cl;
  L.ldy = round_up4(L.mr > 0 ? L.mr : 1);
  L.ldx = round_up4(nJ);
  L.js = (nJ + cl - 1) / cl;
  const size_t small = (size_t)kSmallMats * R * R * 4 + 4 * 32 * 4 + 64;
  size_t off = 0;
  L.off_uc = off;
  off += (size_t)L.mr * ldu * 4;
  L.off_x = off;  // X | Y | Qp | Qs | Qp2 contiguous (zeroed together)
  off += (size_t)R * L.ldx * 4;
  L.off_y = off;
  off += (size_t)R * L.ldy * 4;
  L.off_qp = off;
  off += (size_t)R * L.ldx * 4;
  L.off_qs = off;  // Q = core^T Y, full (every CTA holds the sum of the partials)
  off += (size_t)R * L.ldx * 4;
  L.off_qp2 = off;  // the partials alternate between two buffers from step to step
  off += (size_t)R * L.ldx * 4;
  L.off_end_zero = off;
  L.off_ra = off;
  off += ((size_t)R * R + 4) * 4;
  L.off_ra2 = off;
  off += ((size_t)R * R + 4) * 4;
  L.off_stage = off;  // cl x (R R + 4): remote partials gathered before a fixed-order sum
  off += (size_t)cl * ((size_t)R * R + 4) * 4;
  L.off_slots = off;  // per-warp Cholesky factors
  off += (size_t)(kCsvdThreads / 32) * (R * R + R) * 4;
  L.off_small = off;
  off += small;
  L.off_flag = (off + 15) & ~(size_t)15;
  off = L.off_flag + 16;
  L.off_bar = off;
  off += 16;
  L.total = off;
  return L;
}

size_t csvd_smem_bytes(int nI, int nJ, int Rpad) {
  const CsvdLayout L = csvd_layout(nI, nJ, ld_core(nJ), Rpad, kSvdCluster);
  return L.total > sizeof(SamplerSmem) ? L.total : sizeof(SamplerSmem);
}

// dst[q] = sum over the cluster's CTAs (rank order) of src[q], q < count: the
// kSvdCluster x count remote values are read in parallel into `stage`, then
// every sum is formed in rank order.  Call after a cluster barrier that
// follows every CTA's write of src.
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, float* src, float* dst, int count, float* stage) {
  for (int q = threadIdx.x; q < kSvdCluster * count; q += blockDim.x) {
    const int c = q / count, i = q - c * count;
    stage[q] = cl.map_shared_rank(src, c)[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kSvdCluster; ++c) s += stage[c * count + i];
    dst[i] = s;
  }
  __syncthreads();
}

template <int R>
__device__ __forceinline__ void csvd_body(const IterDesc& d, int role, unsigned char* smem) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  constexpr int ncl = kSvdCluster;
  State* st = d.st;
  if (st->done || st->status) return;  // the same for every CTA: the state is fixed during the launch
  const int k = st->k;
  if (role > 0) {
    // IRCUR-R drawing its own index sets: rank 0 of the clusters of roles 1
    // and 2 draws I_{k+1}, J_{k+1} while the role-0 cluster factorises the core
    const int axis = role - 1;
    if (crank == 0 && d.sampleAhead && k + 1 < d.max_iter) {
      int* out = axis ? const_cast<int*>(d.J_all) + (int64_t)(k + 1) * d.nJ
                      : const_cast<int*>(d.I_all) + (int64_t)(k + 1) * d.nI;
      sample_subset(d.seed, k + 1, axis, axis ? d.n2 : d.n1, axis ? d.nJ : d.nI, out,
                    *reinterpret_cast<SamplerSmem*>(smem));
    }
    return;
  }
  if (crank == 0) trace_start(d.trace, 3 * k + 1);
  const int nI = d.nI, nJ = d.nJ, r = d.r, ldu = d.ldCore;
  const CsvdLayout L = csvd_layout(nI, nJ, ldu, R, ncl);
  const int row0 = crank * L.mr;
  const int nrow = nI - row0 < L.mr ? (nI - row0 > 0 ? nI - row0 : 0) : L.mr;
  const int col0 = crank * L.js;
  const int ncol = nJ - col0 < L.js ? (nJ - col0 > 0 ? nJ - col0 : 0) : L.js;
  float* Uc = reinterpret_cast<float*>(smem + L.off_uc);
  float* X = reinterpret_cast<float*>(smem + L.off_x);
  float* Y = reinterpret_cast<float*>(smem + L.off_y);
  float* Qp0 = reinterpret_cast<float*>(smem + L.off_qp);
  float* Qs = reinterpret_cast<float*>(smem + L.off_qs);
  float* ra0 = reinterpret_cast<float*>(smem + L.off_ra);  // Gram(Y) partials (two buffers)
  float* ra1 = reinterpret_cast<float*>(smem + L.off_ra2);
  float* Qp1 = reinterpret_cast<float*>(smem + L.off_qp2);
  float* stage = reinterpret_cast<float*>(smem + L.off_stage);
  float* slots = reinterpret_cast<float*>(smem + L.off_slots);
  int* flag = reinterpret_cast<int*>(smem + L.off_flag);
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // ---- this CTA's core rows into shared memory: one bulk copy
  const unsigned bytes = (unsigned)((size_t)nrow * ldu * 4);
  if (nrow > 0 && threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(Uc, d.core + (size_t)row0 * ldu, bytes, bar);
  }
  // ---- X, Y, Qp, Qs zeroed (padding rows read as zero); X = B_k(:,J)^T
  {
    const size_t nz = (L.off_end_zero - L.off_x) / 4;
    for (size_t q = threadIdx.x; q < nz; q += blockDim.x) X[q] = 0.f;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
#pragma unroll
    for (int t = 0; t < R; ++t) X[(size_t)t * L.ldx + b] = (t < r) ? d.BJt[(size_t)b * R + t] : 0.f;
  }
  __syncthreads();
  int brk = cholqr_w<R>(X, L.ldx, X, L.ldx, nJ, r, sm.U, sm, slots);
  if (brk > 0) {  // first iteration (B_0 = 0) or a deficient factor: random start
    for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
#pragma unroll
      for (int t = 0; t < R; ++t)
        X[(size_t)t * L.ldx + b] =
            (t < r) ? hash_uniform(d.seed ^ 0x5bd1e995ull, ((uint64_t)k << 32) ^ (uint64_t)(b * R + t)) : 0.f;
    }
    __syncthreads();
    cholqr_w<R>(X, L.ldx, X, L.ldx, nJ, r, sm.U, sm, slots);
  }
  bool ok = true;
  if (nrow > 0) {
    ok = mbar_wait_bounded(bar, 0, d.spinLimit);
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(&st->status, (int)IRCUR_ETIMEOUT);
      mbar_wait_bounded(bar, 0, kSpinLimit);  // let the copy land before the block exits
    }
  }
  ok = __syncthreads_and(ok);
  if (threadIdx.x == 0) *flag = ok ? 0 : 1;
  cl.sync();
  {
    const int mine = threadIdx.x < ncl ? *cl.map_shared_rank(flag, (int)threadIdx.x) : 0;
    if (__syncthreads_or(mine)) {
      cl.sync();  // nobody leaves while others read its flag
      return;
    }
  }

  // ---- subspace iteration.  With Y = (core X) Rp^{-1}, core^T Y =
  // (core^T core X) Rp^{-1}: the transposed product runs on the raw local rows
  // in the same phase as their Gram partial, and Rp^{-1} is applied to the
  // summed Q.  Per step: four block barriers and one cluster barrier (partials
  // written); the partial buffers alternate between steps.
  const int nwarps = (int)(blockDim.x >> 5);
  float* Uw = slots + (size_t)warp * (R * R + R);
  float* dw = Uw + R * R;
  int steps = 0;
  bool converged = false;
  float prev_res = 0.f;
  while (true) {
    ++steps;
    // this step's partial buffers: a CTA that reaches the next step's cluster
    // barrier has finished reading these, so the step after next may reuse them
    float* ra = (steps & 1) ? ra1 : ra0;
    float* Qp = (steps & 1) ? Qp1 : Qp0;
    // Y_c = core_c X (raw): one warp per local row, lanes over the inner index
    for (int o = warp; o < nrow; o += nwarps) {
      float acc[R];
#pragma unroll
      for (int t = 0; t < R; ++t) acc[t] = 0.f;
      for (int q = lane; q < nJ; q += 32) {
        const float u = Uc[(size_t)o * ldu + q];
#pragma unroll
        for (int t = 0; t < R; ++t) acc[t] = fmaf(u, X[(size_t)t * L.ldx + q], acc[t]);
      }
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const float sv = warp_sum(acc[t]);
        if (lane == 0) Y[(size_t)t * L.ldy + o] = sv;
      }
    }
    __syncthreads();
    // Gram(Y_c) partial (one entry per warp) and core_c^T Y_c (one column per thread)
    {
      const int npairs = r * (r + 1) / 2;
      for (int pq = warp; pq < npairs; pq += nwarps) {
        int s0 = 0, rem = pq;
        while (rem >= r - s0) {
          rem -= r - s0;
          ++s0;
        }
        const int t1 = s0 + rem;
        float acc = 0.f;
        for (int i = lane; i < nrow; i += 32) acc = fmaf(Y[(size_t)s0 * L.ldy + i], Y[(size_t)t1 * L.ldy + i], acc);
        acc = warp_sum(acc);
        if (lane == 0) {
          ra[s0 * R + t1] = acc;
          ra[t1 * R + s0] = acc;
        }
      }
      for (int j = threadIdx.x; j < nJ; j += blockDim.x) {
        float acc[R];
#pragma unroll
        for (int t = 0; t < R; ++t) acc[t] = 0.f;
        for (int i = 0; i < nrow; ++i) {
          const float u = Uc[(size_t)i * ldu + j];
#pragma unroll
          for (int t = 0; t < R; ++t) acc[t] = fmaf(u, Y[(size_t)t * L.ldy + i], acc[t]);
        }
#pragma unroll
        for (int t = 0; t < R; ++t) Qp[(size_t)t * L.ldx + j] = acc[t];
      }
    }
    cl.sync();  // (1) partials written
    // the cluster sums, rank order: Gram(Y) and Q = core^T Y_raw
    for (int q = threadIdx.x; q < R * R; q += blockDim.x) {
      float v[ncl];
#pragma unroll
      for (int c = 0; c < ncl; ++c) v[c] = cl.map_shared_rank(ra, c)[q];
      float sacc = 0.f;
#pragma unroll
      for (int c = 0; c < ncl; ++c) sacc += v[c];
      sm.G[q] = sacc;
    }
    for (int q = threadIdx.x; q < R * nJ; q += blockDim.x) {
      const int t = q / nJ, b = q - t * nJ;
      const size_t at = (size_t)t * L.ldx + b;
      float v[ncl];
#pragma unroll
      for (int c = 0; c < ncl; ++c) v[c] = cl.map_shared_rank(Qp, c)[at];  // all in flight
      float sacc = 0.f;
#pragma unroll
      for (int c = 0; c < ncl; ++c) sacc += v[c];
      Qs[at] = sacc;
    }
    __syncthreads();  // the sums are visible to the whole block
    // Y Rp = core X: every warp factorises Gram(Y); Q = Q_raw Rp^{-1} row by
    // row, with the residual ||Q - X Rp^T||_F^2 of each row
    {
      float* Up = warp == 0 ? sm.Rp : Uw;
      float* dp = warp == 0 ? sm.dinv : dw;
      warp_chol<R>(sm.G, r, Up, dp);
      float e2 = 0.f;
      for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
        float m[R], y[R], xr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
          m[t] = Qs[(size_t)t * L.ldx + b];
          xr[t] = X[(size_t)t * L.ldx + b];
        }
        row_subst<R>(m, y, Up, dp);
#pragma unroll
        for (int t = 0; t < R; ++t) {
          Qs[(size_t)t * L.ldx + b] = y[t];
          float v = y[t];
#pragma unroll
          for (int s2 = t; s2 < R; ++s2) v = fmaf(-xr[s2], Up[t * R + s2], v);
          e2 = fmaf(v, v, e2);
        }
      }
      e2 = warp_sum(e2);
      if (lane == 0) sm.red[warp] = e2;
    }
    __syncthreads();
    float E2 = 0.f;
    for (int w = 0; w < nwarps; ++w) E2 += sm.red[w];
    float RC2 = 0.f;  // ||Rp||_F^2 = trace Gram(Y)
#pragma unroll
    for (int t = 0; t < R; ++t) RC2 += sm.G[t * R + t];
    const float res = sqrtf(E2), nrm = sqrtf(RC2);
    if (res <= 1e-6f * nrm || (steps > 1 && res > 0.5f * prev_res && res <= 1e-5f * nrm) || !(nrm > 0.f)) {
      converged = true;
      break;
    }
    if (steps >= d.svdMaxSteps) break;  // keep X, Y, Rp of the same step
    prev_res = res;
    cholqr_w<R>(Qs, L.ldx, X, L.ldx, nJ, r, sm.U, sm, slots);  // X = orth(core^T Y), in every CTA
  }
  // Y of the last step: Y = (core X) Rp^{-1}
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) {
    float m[R], y[R];
#pragma unroll
    for (int t = 0; t < R; ++t) m[t] = Y[(size_t)t * L.ldy + i];
    row_subst<R>(m, y, sm.Rp, sm.dinv);
#pragma unroll
    for (int t = 0; t < R; ++t) Y[(size_t)t * L.ldy + i] = y[t];
  }
  __syncthreads();

  // ---- second CholQR passes (Y over the cluster, X replicated); T = U2y Rp U2x^{-1}
  float* raF = (steps & 1) ? ra0 : ra1;  // not the last step's buffer (others may still read that)
  gram_block<R>(Y, nrow, L.ldy, r, raF);
  cl.sync();
  cluster_sum(cl, raF, sm.G, R * R, stage);
  {
    float* Up = warp == 0 ? sm.U2y : Uw;
    float* dp = warp == 0 ? sm.dinv : dw;
    warp_chol<R>(sm.G, r, Up, dp);
    for (int i = threadIdx.x; i < nrow; i += blockDim.x) {
      float m[R], y[R];
#pragma unroll
      for (int t = 0; t < R; ++t) m[t] = Y[(size_t)t * L.ldy + i];
      row_subst<R>(m, y, Up, dp);
#pragma unroll
      for (int t = 0; t < R; ++t) Y[(size_t)t * L.ldy + i] = y[t];
    }
  }
  __syncthreads();
  cholqr_w<R>(X, L.ldx, X, L.ldx, nJ, r, sm.U2x, sm, slots);
  if (threadIdx.x < 32) {
    const int s2 = threadIdx.x;
    if (s2 < r) {
      float row[R];  // (U2y Rp)(s2, :)
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = 0.f;
        for (int u = 0; u < r; ++u) v = fmaf(sm.U2y[s2 * R + u], sm.Rp[u * R + t], v);
        row[t] = v;
      }
      float tr[R];  // T(s2,:) U2x = row (forward substitution; dropped pivots give zeros)
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = row[t];
#pragma unroll
        for (int u = 0; u < t; ++u) v = fmaf(-tr[u], sm.U2x[u * R + t], v);
        tr[t] = (t < r) ? v * sm.dinv[t] : 0.f;
      }
#pragma unroll
      for (int t = 0; t < R; ++t) sm.T[s2 * R + t] = tr[t];
    }
  }
  __syncthreads();
  // ---- numerical rank from the diagonal of T, and T^{-1} on the kept pivots
  if (warp == 0) {
    const float dabs = lane < r ? fabsf(sm.T[lane * R + lane]) : 0.f;
    float dmax = dabs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    const float tol = (float)(nI > nJ ? nI : nJ) * FLT_EPSILON * dmax;
    const bool keep = lane < r && dabs > tol && dabs > 0.f;
    const unsigned kmask = __ballot_sync(0xffffffffu, keep);
    if (lane < r) {
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
      for (int s2 = 0; s2 < R; ++s2) sm.Ut[s2 * R + c] = x[s2];
      sm.sig[lane] = keep ? dabs : 0.f;
    }
    if (lane == 0) {
      sm.ibuf[1] = __popc(kmask);
      sm.ibuf[2] = (int)kmask;
      for (int t = r; t < R; ++t) {
        sm.sig[t] = 0.f;
        for (int u = 0; u < R; ++u) sm.Ut[u * R + t] = 0.f;
      }
    }
  }
  __syncthreads();
  const int rank = sm.ibuf[1];
  const unsigned kmask = (unsigned)sm.ibuf[2];
  // Outputs (U^+ = X T^{-1} Y^T): W = Y by this CTA's rows; Vs = X T^{-1} and
  // V = X T^T by this CTA's slice.
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) {
#pragma unroll
    for (int t = 0; t < R; ++t)
      d.W[(size_t)(row0 + i) * R + t] = ((kmask >> t) & 1u) ? Y[(size_t)t * L.ldy + i] : 0.f;
  }
  for (int bb = threadIdx.x; bb < ncol; bb += blockDim.x) {
    const int b = col0 + bb;
    float x[R];
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) x[s2] = X[(size_t)s2 * L.ldx + b];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float vp = 0.f, vr = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) {
        vp = fmaf(x[s2], sm.Ut[s2 * R + t], vp);
        vr = fmaf(x[s2], sm.T[t * R + s2], vr);
      }
      const bool kt = (kmask >> t) & 1u;
      d.Vs[(size_t)b * R + t] = kt ? vp : 0.f;
      d.V[(size_t)b * R + t] = kt ? vr : 0.f;
    }
  }
  if (crank == 0) {
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
  }
  cl.sync();  // no CTA leaves while another may still read its shared memory
  if (crank == 0 && d.trace) {
    __syncthreads();
    trace_stop(d.trace, 3 * d.max_iter, 3 * k + 1);
  }
}

// Up to R = 7 the cluster SVD fits in 128 registers without spilling; the
// cap leaves room on its SMs for the pass blocks that start while it runs.
template <int R>
__global__ void __launch_bounds__(kCsvdThreads, (R <= 7 ? 2 : 1)) csvd_kernel(IterDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  // every CTA is resident from here on: the pass kernel may start on the
  // other SMs (it waits for this grid before reading its outputs)
  pdl_launch_dependents();
  csvd_body<R>(d, blockIdx.y, smem);
}

// Batched form: cluster blockIdx.x / kSvdCluster factorises instance
// list[blockIdx.x / kSvdCluster]; blockIdx.y is the role.
template <int R>
__global__ void __launch_bounds__(kCsvdThreads, (R <= 7 ? 2 : 1)) csvd_batch_kernel(const IterDesc* __restrict__ ds,
                                                                    const int* __restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_launch_dependents();  // the batched pass kernel may start (it waits before the projections)
  csvd_body<R>(ds[list[blockIdx.x / kSvdCluster]], blockIdx.y, smem);
}

// ---------------------------------------------------------------------------
// Core SVD in one CTA, for cores that fit in one SM's shared memory (R <= 8,
// where the padded rank equals r).  The same two-sided subspace iteration,
// warm start and stopping rule as the cluster form above, with every
// exchange inside one block of 1024 threads instead of across a cluster:
//   P  = core X      threads (row i, column segment s) sum 16-byte column
//                    quads of their row; thread i adds the segments in order
//                    and forms its row's Gram(P) products
//   Q~ = core^T P    threads (column quad q, row segment s), the same way
//   Rp = chol(Gram P), Q = Q~ Rp^{-1}, the residual Q - X Rp^T and the
//                    Gram(Q) products by thread j (Q stays in its registers)
//   X  = Q chol(Gram Q)^{-1}
// Factors of the r x r Gram matrices are formed redundantly by every warp
// that owns rows, so the rows they transform need no further barrier: five
// block barriers per step.  Every sum runs in a fixed order (bit-identical
// results from launch to launch).
constexpr int kSsvdThreads = 1024;
constexpr int kSsvdMaxR = 8;
constexpr int kSsvdSeg = 8;  // most segments of either partial product

__host__ __device__ constexpr int npairs_of(int R) { return R * (R + 1) / 2; }

struct SsvdLayout {
  int nq;       // 16-byte column quads of the core, ceil(nJ / 4)
  int ldx;      // column stride of X and of the core^T P partials (4 nq)
  int ldy;      // column stride of the P partials (nI rounded up to 4)
  int ps;       // row stride of P (R rounded up to 4)
  int s1, qs1;  // P partials: column segments, quads per segment
  int s3, rs3;  // core^T P partials: row segments, rows per segment
  int nw;       // warps owning rows, ceil(max(nI, nJ) / 32)
  int slot;     // floats per warp slot
  size_t off_uc, off_x, off_p, off_part, off_red, off_slots, off_flag, off_bar, total;
};

__host__ __device__ inline SsvdLayout ssvd_layout(int nI, int nJ, int ldu, int R) {
  SsvdLayout L;
  const int nt = kSsvdThreads;
  L.nq = (nJ + 3) / 4;
  L.ldx = 4 * L.nq;
  L.ldy = round_up4(nI);
  L.ps = round_up4(R);
  L.s1 = nt / (nI > 0 ? nI : 1);
  L.s1 = L.s1 < 1 ? 1 : (L.s1 > kSsvdSeg ? kSsvdSeg : L.s1);
  L.qs1 = (L.nq + L.s1 - 1) / L.s1;
  L.s3 = nt / (L.nq > 0 ? L.nq : 1);
  L.s3 = L.s3 < 1 ? 1 : (L.s3 > kSsvdSeg ? kSsvdSeg : L.s3);
  L.rs3 = (nI + L.s3 - 1) / L.s3;
  const int mx = nI > nJ ? nI : nJ;
  L.nw = (mx + 31) / 32;
  L.slot = 6 * R * R + 3 * R;
  const size_t part = (size_t)R * ((size_t)L.s1 * L.ldy > (size_t)L.s3 * L.ldx ? (size_t)L.s1 * L.ldy
                                                                               : (size_t)L.s3 * L.ldx);
  size_t off = 0;
  L.off_uc = off;
  off += (size_t)nI * ldu * 4;
  L.off_x = off;
  off += (size_t)R * L.ldx * 4;
  L.off_p = off;
  off += (size_t)nI * L.ps * 4;
  L.off_part = off;
  off += part * 4;
  L.off_red = off;  // per warp: Gram pairs (two sets) and one residual sum
  off += (size_t)L.nw * (2 * npairs_of(R) + 1) * 4;
  L.off_slots = off;
  off += (size_t)L.nw * L.slot * 4;
  L.off_flag = (off + 15) & ~(size_t)15;
  off = L.off_flag + 16;
  L.off_bar = off;
  off += 16;
  L.total = off;
  return L;
}

size_t ssvd_smem_bytes(int nI, int nJ, int Rpad) {
  if (Rpad > kSsvdMaxR || nI > kSsvdThreads || nJ > kSsvdThreads || nI < 1 || nJ < 1) return ~(size_t)0;
  const SsvdLayout L = ssvd_layout(nI, nJ, ld_core(nJ), Rpad);
  return L.total > sizeof(SamplerSmem) ? L.total : sizeof(SamplerSmem);
}

bool ssvd_fits(int nI, int nJ, int Rpad) { return ssvd_smem_bytes(nI, nJ, Rpad) <= 227 * 1024; }

// The Gram products of one row (a) summed over the warp; lane 0 writes the
// R(R+1)/2 upper-triangle sums to out.
template <int R>
__device__ __forceinline__ void warp_pair_sums(const float (&a)[R], float* out) {
  int p = 0;
#pragma unroll
  for (int s0 = 0; s0 < R; ++s0) {
#pragma unroll
    for (int t1 = s0; t1 < R; ++t1) {
      const float v = warp_sum(a[s0] * a[t1]);
      if ((threadIdx.x & 31) == 0) out[p] = v;
      ++p;
    }
  }
}

// Gw = the sum over warps 0..nw-1 (in order) of their pair sums, both triangles.
template <int R>
__device__ __forceinline__ void gram_from_pairs(const float* red, int stride, int nw, float* Gw) {
  const int lane = threadIdx.x & 31;
  constexpr int np = npairs_of(R);
  for (int p = lane; p < np; p += 32) {
    float v = 0.f;
    for (int w = 0; w < nw; ++w) v += red[w * stride + p];
    int s0 = 0, rem = p;
    while (rem >= R - s0) {
      rem -= R - s0;
      ++s0;
    }
    const int t1 = s0 + rem;
    Gw[s0 * R + t1] = v;
    Gw[t1 * R + s0] = v;
  }
  __syncwarp();
}

template <int R>
__device__ __forceinline__ void ssvd_body(const IterDesc& d, int role, unsigned char* smem) {
  static_assert(R <= kSsvdMaxR, "one-CTA core SVD is built for R <= 8");
  State* st = d.st;
  if (st->done || st->status) return;  // the same for every thread: the state is fixed during the launch
  const int k = st->k;
  if (role > 0) {
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
  const int nI = d.nI, nJ = d.nJ, ldu = d.ldCore;
  constexpr int np = npairs_of(R);
  const SsvdLayout L = ssvd_layout(nI, nJ, ldu, R);
  float* Uc = reinterpret_cast<float*>(smem + L.off_uc);
  float* X = reinterpret_cast<float*>(smem + L.off_x);
  float* P = reinterpret_cast<float*>(smem + L.off_p);
  float* part = reinterpret_cast<float*>(smem + L.off_part);
  float* redA = reinterpret_cast<float*>(smem + L.off_red);  // nw x np
  float* redB = redA + (size_t)L.nw * np;                     // nw x np
  float* redE = redB + (size_t)L.nw * np;                     // nw
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.off_bar);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool rowwarp = warp < L.nw;
  // this warp's slot: Gram scratch, Rp (+ reciprocal pivots), Uq / U2y, U2x, T, T^{-1}
  float* Gw = reinterpret_cast<float*>(smem + L.off_slots) + (size_t)(rowwarp ? warp : 0) * L.slot;
  float* Rpw = Gw + R * R;
  float* dRp = Rpw + R * R;
  float* Uqw = dRp + R;
  float* dUq = Uqw + R * R;
  float* U2x = dUq + R;
  float* dU2x = U2x + R * R;
  float* Tw = dU2x + R;
  float* Utw = Tw + R * R;

  // ---- the core into shared memory: one bulk copy
  const unsigned bytes = (unsigned)((size_t)nI * ldu * 4);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, bytes);
    bulk_g2s(Uc, d.core, bytes, bar);
  }
  for (int q = tid; q < R * L.ldx; q += blockDim.x) X[q] = 0.f;
  // ---- X = orth(B_k(:,J)^T), or a random start when that is deficient
  float xb[R];
#pragma unroll
  for (int t = 0; t < R; ++t) xb[t] = (tid < nJ) ? d.BJt[(size_t)tid * R + t] : 0.f;
  if (rowwarp) warp_pair_sums<R>(xb, redB + warp * np);
  __syncthreads();
  int brk = 0;
  if (rowwarp) {
    gram_from_pairs<R>(redB, np, L.nw, Gw);
    brk = warp_chol<R>(Gw, R, Uqw, dUq);
    if (brk == 0) {
      if (tid < nJ) {
        float y[R];
        row_subst<R>(xb, y, Uqw, dUq);
#pragma unroll
        for (int t = 0; t < R; ++t) X[(size_t)t * L.ldx + tid] = y[t];
      }
    } else {
#pragma unroll
      for (int t = 0; t < R; ++t)
        xb[t] = (tid < nJ)
                    ? hash_uniform(d.seed ^ 0x5bd1e995ull, ((uint64_t)k << 32) ^ (uint64_t)(tid * R + t))
                    : 0.f;
      warp_pair_sums<R>(xb, redA + warp * np);
    }
  }
  __syncthreads();
  if (rowwarp && brk > 0) {  // brk is the same in every row warp
    gram_from_pairs<R>(redA, np, L.nw, Gw);
    warp_chol<R>(Gw, R, Uqw, dUq);
    if (tid < nJ) {
      float y[R];
      row_subst<R>(xb, y, Uqw, dUq);
#pragma unroll
      for (int t = 0; t < R; ++t) X[(size_t)t * L.ldx + tid] = y[t];
    }
  }
  bool ok = mbar_wait_bounded(bar, 0, d.spinLimit);
  if (!ok) {
    if (tid == 0) atomicExch(&st->status, (int)IRCUR_ETIMEOUT);
    mbar_wait_bounded(bar, 0, kSpinLimit);  // let the copy land before the block exits
  }
  if (!__syncthreads_and(ok)) return;
  // columns nJ .. 4 nq of the last quad read as zero
  for (int q = tid; q < nI * (L.ldx - nJ); q += blockDim.x) {
    const int i = q / (L.ldx - nJ), c = nJ + q % (L.ldx - nJ);
    Uc[(size_t)i * ldu + c] = 0.f;
  }
  __syncthreads();

  // ---- subspace iteration
  const int seg1 = tid / nI, i1 = tid - seg1 * nI;      // P partials
  const int seg3 = tid / L.nq, q3 = tid - seg3 * L.nq;  // core^T P partials
  int steps = 0;
  bool converged = false;
  float prev_res = 0.f;
  float qv[R];
  while (true) {
    ++steps;
    if (seg1 < L.s1) {
      float acc[R];
#pragma unroll
      for (int t = 0; t < R; ++t) acc[t] = 0.f;
      const int qa = seg1 * L.qs1, qb = qa + L.qs1 < L.nq ? qa + L.qs1 : L.nq;
      const float* urow = Uc + (size_t)i1 * ldu;
      for (int q = qa; q < qb; ++q) {
        const float4 u = *reinterpret_cast<const float4*>(urow + 4 * q);
#pragma unroll
        for (int t = 0; t < R; ++t) {
          const float4 x = *reinterpret_cast<const float4*>(X + (size_t)t * L.ldx + 4 * q);
          acc[t] = fmaf(u.x, x.x, acc[t]);
          acc[t] = fmaf(u.y, x.y, acc[t]);
          acc[t] = fmaf(u.z, x.z, acc[t]);
          acc[t] = fmaf(u.w, x.w, acc[t]);
        }
      }
#pragma unroll
      for (int t = 0; t < R; ++t) part[(size_t)(seg1 * R + t) * L.ldy + i1] = acc[t];
    }
    __syncthreads();
    if (rowwarp) {
      float pv[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = 0.f;
        if (tid < nI)
          for (int s = 0; s < L.s1; ++s) v += part[(size_t)(s * R + t) * L.ldy + tid];
        pv[t] = v;
      }
      if (tid < nI) {
#pragma unroll
        for (int t = 0; t < R; ++t) P[(size_t)tid * L.ps + t] = pv[t];
      }
      warp_pair_sums<R>(pv, redA + warp * np);
    }
    __syncthreads();
    if (seg3 < L.s3) {
      float acc[4][R];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int t = 0; t < R; ++t) acc[c][t] = 0.f;
      const int ia = seg3 * L.rs3, ib = ia + L.rs3 < nI ? ia + L.rs3 : nI;
      for (int i = ia; i < ib; ++i) {
        const float4 u = *reinterpret_cast<const float4*>(Uc + (size_t)i * ldu + 4 * q3);
        const float4* prow = reinterpret_cast<const float4*>(P + (size_t)i * L.ps);
        const float4 pa = prow[0];
        const float4 pb = (R > 4) ? prow[1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float pall[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
        float pr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) pr[t] = pall[t];
#pragma unroll
        for (int t = 0; t < R; ++t) {
          acc[0][t] = fmaf(u.x, pr[t], acc[0][t]);
          acc[1][t] = fmaf(u.y, pr[t], acc[1][t]);
          acc[2][t] = fmaf(u.z, pr[t], acc[2][t]);
          acc[3][t] = fmaf(u.w, pr[t], acc[3][t]);
        }
      }
#pragma unroll
      for (int t = 0; t < R; ++t)
        *reinterpret_cast<float4*>(part + (size_t)(seg3 * R + t) * L.ldx + 4 * q3) =
            make_float4(acc[0][t], acc[1][t], acc[2][t], acc[3][t]);
    }
    __syncthreads();
    if (rowwarp) {
      // Rp: Y Rp = P (Y = P Rp^{-1} is never formed inside the loop)
      gram_from_pairs<R>(redA, np, L.nw, Gw);
      warp_chol<R>(Gw, R, Rpw, dRp);
      float e2 = 0.f;
#pragma unroll
      for (int t = 0; t < R; ++t) qv[t] = 0.f;
      if (tid < nJ) {
        float m[R], xr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
          float v = 0.f;
          for (int s = 0; s < L.s3; ++s) v += part[(size_t)(s * R + t) * L.ldx + tid];
          m[t] = v;
          xr[t] = X[(size_t)t * L.ldx + tid];
        }
        row_subst<R>(m, qv, Rpw, dRp);  // Q = core^T Y
#pragma unroll
        for (int t = 0; t < R; ++t) {
          float v = qv[t];
#pragma unroll
          for (int s2 = t; s2 < R; ++s2) v = fmaf(-xr[s2], Rpw[t * R + s2], v);
          e2 = fmaf(v, v, e2);
        }
      }
      warp_pair_sums<R>(qv, redB + warp * np);
      e2 = warp_sum(e2);
      if (lane == 0) redE[warp] = e2;
    }
    __syncthreads();
    // the same decision in every thread: sums over the row warps in order
    float E2 = 0.f, RC2 = 0.f;
    for (int w = 0; w < L.nw; ++w) E2 += redE[w];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int pd = t * R - t * (t - 1) / 2;  // pair (t, t)
      float g = 0.f;
      for (int w = 0; w < L.nw; ++w) g += redA[w * np + pd];
      RC2 += g;  // ||Rp||_F^2 = trace Gram(P)
    }
    const float res = sqrtf(E2), nrm = sqrtf(RC2);
    if (res <= 1e-6f * nrm || (steps > 1 && res > 0.5f * prev_res && res <= 1e-5f * nrm) || !(nrm > 0.f)) {
      converged = true;
      break;
    }
    if (steps >= d.svdMaxSteps) break;  // keep X, P, Rp of the same step
    prev_res = res;
    if (rowwarp) {
      gram_from_pairs<R>(redB, np, L.nw, Gw);
      warp_chol<R>(Gw, R, Uqw, dUq);
      if (tid < nJ) {
        float y[R];
        row_subst<R>(qv, y, Uqw, dUq);
#pragma unroll
        for (int t = 0; t < R; ++t) X[(size_t)t * L.ldx + tid] = y[t];
      }
    }
    __syncthreads();
  }

  // ---- Y = P Rp^{-1}; second CholQR passes of Y and X; T = U2y Rp U2x^{-1}
  float yv[R], xv[R];
  if (rowwarp) {
    {
      float m[R];
#pragma unroll
      for (int t = 0; t < R; ++t) m[t] = (tid < nI) ? P[(size_t)tid * L.ps + t] : 0.f;
      row_subst<R>(m, yv, Rpw, dRp);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) xv[t] = (tid < nJ) ? X[(size_t)t * L.ldx + tid] : 0.f;
    warp_pair_sums<R>(yv, redA + warp * np);
    warp_pair_sums<R>(xv, redB + warp * np);
  }
  __syncthreads();
  if (rowwarp) {
    gram_from_pairs<R>(redA, np, L.nw, Gw);
    warp_chol<R>(Gw, R, Uqw, dUq);  // U2y
    gram_from_pairs<R>(redB, np, L.nw, Gw);
    warp_chol<R>(Gw, R, U2x, dU2x);
    if (lane < R) {
      const int s2 = lane;
      float row[R];  // (U2y Rp)(s2, :)
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = 0.f;
#pragma unroll
        for (int u = 0; u < R; ++u) v = fmaf(Uqw[s2 * R + u], Rpw[u * R + t], v);
        row[t] = v;
      }
      float tr[R];  // T(s2,:) U2x = row (forward substitution; dropped pivots give zeros)
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float v = row[t];
#pragma unroll
        for (int u = 0; u < t; ++u) v = fmaf(-tr[u], U2x[u * R + t], v);
        tr[t] = v * dU2x[t];
      }
#pragma unroll
      for (int t = 0; t < R; ++t) Tw[s2 * R + t] = tr[t];
    }
    __syncwarp();
    // numerical rank from the diagonal of T, and T^{-1} on the kept pivots
    const float dabs = lane < R ? fabsf(Tw[lane * R + lane]) : 0.f;
    float dmax = dabs;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    const float tol = (float)(nI > nJ ? nI : nJ) * FLT_EPSILON * dmax;
    const bool keep = lane < R && dabs > tol && dabs > 0.f;
    const unsigned kmask = __ballot_sync(0xffffffffu, keep);
    if (lane < R) {
      const int c = lane;
      float x[R];
#pragma unroll
      for (int s2 = R - 1; s2 >= 0; --s2) {
        float v = 0.f;
        if (s2 <= c && ((kmask >> s2) & 1u)) {
          v = (s2 == c) ? 1.f : 0.f;
#pragma unroll
          for (int u = s2 + 1; u < R; ++u)
            if (u <= c) v = fmaf(-Tw[s2 * R + u], x[u], v);
          v = v / Tw[s2 * R + s2];
        }
        x[s2] = v;
      }
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) Utw[s2 * R + c] = x[s2];
    }
    __syncwarp();
    // outputs (U^+ = X T^{-1} Y^T): W = Y; Vs = X T^{-1}; V = X T^T
    if (tid < nI) {
      float y2[R];
      row_subst<R>(yv, y2, Uqw, dUq);
#pragma unroll
      for (int t = 0; t < R; ++t) d.W[(size_t)tid * R + t] = ((kmask >> t) & 1u) ? y2[t] : 0.f;
    }
    if (tid < nJ) {
      float x2[R];
      row_subst<R>(xv, x2, U2x, dU2x);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        float vp = 0.f, vr = 0.f;
#pragma unroll
        for (int s2 = 0; s2 < R; ++s2) {
          vp = fmaf(x2[s2], Utw[s2 * R + t], vp);
          vr = fmaf(x2[s2], Tw[t * R + s2], vr);
        }
        const bool kt = (kmask >> t) & 1u;
        d.Vs[(size_t)tid * R + t] = kt ? vp : 0.f;
        d.V[(size_t)tid * R + t] = kt ? vr : 0.f;
      }
    }
    if (warp == 0) {
      if (lane < R) d.sigma[lane] = keep ? dabs : 0.f;
      for (int q = lane; q < R * R; q += 32) d.Tm[q] = Tw[q];
      if (lane == 0) {
        unsigned f = 0u;
        if (__popc(kmask) < R) f |= IRCUR_FLAG_WRANK;
        if (!converged) f |= IRCUR_FLAG_SVD_NOCONV;
        if (f) atomicOr(&st->flags, f);
        st->svd_steps += steps;
        st->svd_last_steps = steps;
      }
    }
  }
  if (d.trace) {
    __syncthreads();
    trace_stop(d.trace, 3 * d.max_iter, 3 * k + 1);
  }
}

template <int R>
__global__ void __launch_bounds__(kSsvdThreads, 1) ssvd_kernel(IterDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_launch_dependents();
  ssvd_body<R>(d, blockIdx.y, smem);
}

// Batched form: block x factorises instance list[x]; blockIdx.y is the role.
template <int R>
__global__ void __launch_bounds__(kSsvdThreads, 1) ssvd_batch_kernel(const IterDesc* __restrict__ ds,
                                                                    const int* __restrict__ list) {
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_launch_dependents();
  ssvd_body<R>(ds[list[blockIdx.x]], blockIdx.y, smem);
}

template <typename... Args>
static cudaError_t launch_cluster(void (*kernel)(Args...), dim3 grid, size_t smem, cudaStream_t s,
                                  Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // the largest shared-memory carveout on the SVD's SMs, so that the pass
  // blocks launched while it runs fit next to it
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kCsvdThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kSvdCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int R>
static cudaError_t launch_csvd_r(const IterDesc& d, cudaStream_t s) {
  const size_t bytes = csvd_smem_bytes(d.nI, d.nJ, R);
  return launch_cluster(csvd_kernel<R>, dim3(kSvdCluster, 1 + (d.sampleAhead ? 2 : 0), 1), bytes, s, d);
}

template <int R>
static cudaError_t launch_csvd_batch_r(const BatchLaunch& b, cudaStream_t s) {
  const int n = b.svd_n[1];
  if (n == 0) return cudaSuccess;
  return launch_cluster(csvd_batch_kernel<R>, dim3(kSvdCluster * n, b.svd_roles, 1), b.svd_smem[1], s, b.ds,
                        b.svd_list[1]);
}

template <int R>
static cudaError_t launch_ssvd_r(const IterDesc& d, cudaStream_t s) {
  if constexpr (R > kSsvdMaxR) {
    return cudaErrorInvalidValue;
  } else {
    const size_t bytes = ssvd_smem_bytes(d.nI, d.nJ, R);
    cudaError_t e = cudaFuncSetAttribute(ssvd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ssvd_kernel<R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    ssvd_kernel<R><<<dim3(1, 1 + (d.sampleAhead ? 2 : 0), 1), kSsvdThreads, bytes, s>>>(d);
    return cudaGetLastError();
  }
}

template <int R>
static cudaError_t launch_ssvd_batch_r(const BatchLaunch& b, cudaStream_t s) {
  if constexpr (R > kSsvdMaxR) {
    return b.svd_n[0] ? cudaErrorInvalidValue : cudaSuccess;
  } else {
    const int n = b.svd_n[0];
    if (n == 0) return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(ssvd_batch_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.svd_smem[0]);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ssvd_batch_kernel<R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    ssvd_batch_kernel<R><<<dim3(n, b.svd_roles, 1), kSsvdThreads, b.svd_smem[0], s>>>(b.ds, b.svd_list[0]);
    return cudaGetLastError();
  }
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
  if (d.svdOneCta) return launch_ssvd_r<R>(d, s);
  return launch_csvd_r<R>(d, s);
}

template <int R>
static cudaError_t launch_svd_batch_r(const BatchLaunch& b, cudaStream_t s) {
  cudaError_t e = launch_ssvd_batch_r<R>(b, s);
  if (e != cudaSuccess) return e;
  return launch_csvd_batch_r<R>(b, s);
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
