// The core of one IRCUR iteration (Alg. 1): Phase I on the |I| x |J| block,
//   core = [D - S_{k+1}]_{I,J},  S_{k+1} = T_zeta(D - L_k)   (Sec. 3.2),
// and Phase II, the rank-r truncation U_{k+1} = H_r(core) with its
// pseudo-inverse U^+ = V_r Sigma_r^{-1} W_r^T (Sec. 3.1), on one thread-block
// cluster of NC CTAs (NC = 1 .. 16).
//
// Core.  L_k(I,J) = A_k(I,:) B_k(:,J) is evaluated entry by entry with the
// same FMA chain as the panel passes (lowrank_entry), so the core equals the
// (I,J) entries of both panels bit for bit.  D(I,J) comes from a compact copy
// (row-major), loaded by bulk copies.  CTA c holds the core rows [c mI/NC, ...)
// (row slab, for core X) and the core columns [c mJ/NC, ...) (column slab,
// stored transposed, for core^T Y) in shared memory.  Each entry is formed
// once, by the owner of its row, and pushed to the owner of its column; with
// NC = 1 one copy with an odd leading dimension serves both products
// conflict-free.
//
// Truncation.  Two-sided subspace iteration, warm-started from B_k(:,J)^T, the
// right factor of the previous iterate on the new columns (close to the
// previous core's X T^T, nearly orthogonal columns graded by T's diagonal),
// with its columns divided by |T_tt|.  Half-steps alternate:
//   P  = core X            (row slabs)   Y Rp = P    (Cholesky QR, Y replaces P)
//   Q  = core^T Y          (column slabs) X Uq = Q   (Cholesky QR, X replaces Q)
// Each half-step ends with one all-gather over distributed shared memory: every
// CTA pushes its rows of P (or Q) and its partial Gram matrix to every CTA,
// then one cluster barrier; the r x r Cholesky factors are formed redundantly
// by every warp from the partials summed in rank order, so every warp of every
// CTA holds bit-identical factors and takes identical branch decisions.
// Convergence is tested after every half-step on the residual of the pair it
// completes: after P, ||core X - Y_prev Uq^T|| (left); after Q,
// ||core^T Y - X Rp^T|| (right).  The test is scaled by 1 - rho, rho the
// residual's contraction per half-step (an estimate of sigma_{r+1}/sigma_r),
// so a narrow gap iterates until the truncated subspace itself is accurate, not
// only the residual; a residual that stops shrinking has reached the FP32
// floor (IRCUR_FLAG_SVD_GAP if the target was not met), a step cap ends the
// rest (IRCUR_FLAG_SVD_NOCONV).
//
// Accuracy.  Cholesky QR in FP32 is accurate when the scaled Gram matrix
// D^{-1/2} G D^{-1/2} is well conditioned, which the graded warm start gives.
// When a scaled pivot shows that FP32 cancellation could ruin the factor
// (pivot / G_tt < 1e-4: an unaligned basis of an ill-conditioned core), the
// Gram matrix of the gathered block is formed again in FP64 and factorised in
// FP64, and the basis is rotated to Ritz vectors (one-warp Jacobi SVD of the
// r x r factor) so that the following half-steps are graded again.
//
// Output.  At convergence the pair (Y, X) and T = Y^T core X (Rp, or Uq^T) give
// H_r(core) = Y T X^T; a one-warp Jacobi SVD T = Ut Sigma Vt^T yields the
// singular values (numerical rank: sigma_i > max(|I|,|J|) * FLT_EPSILON * sigma_1,
// else IRCUR_FLAG_WRANK) and the outputs in the Ritz basis:
//   W = Y Ut (left singular vectors), Vs = X Vt Sigma^{-1}, V = X Vt Sigma,
// so U^+ = Vs W^T, and the next iteration's warm start is graded.
#pragma once

#include <cooperative_groups.h>
#include <float.h>
#include <string.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"
#include "sampler.cuh"

namespace ircur {

namespace cg = cooperative_groups;

__host__ __device__ constexpr int svd_np(int R) { return R * (R + 1) / 2; }
__host__ __device__ constexpr int svd_pow2(int x) { return x <= 1 ? 1 : 2 * svd_pow2((x + 1) / 2); }
// rows of one product group: G R <= 16 partial sums per lane, reduced together
__host__ __device__ constexpr int svd_gmax(int R) { return (16 / R) < 1 ? 1 : (16 / R); }
// largest cluster: loops over the cluster's CTAs are unrolled to this bound
constexpr int kSvdMaxNC = 16;
// replicated factors (every warp its own copy) up to R = 10; one shared copy above
__host__ __device__ constexpr bool svd_rep(int R) { return R <= 10; }
__host__ __device__ constexpr int svd_slot(int R) { return (svd_np(R) + 2 + 3) & ~3; }
__host__ __device__ constexpr int svd_wslot(int R) { return (3 * R * R + 2 * R + 4 + 3) & ~3; }

constexpr int kSvdThreadsCl = 256;   // threads per CTA of a cluster form (NC > 1)
constexpr int kSvdThreadsOne = 512;  // threads of the one-CTA form (NC = 1)
constexpr float kPivotFp64 = 1e-4f;  // scaled Cholesky pivot below which the factor is redone in FP64
constexpr float kRegrade = 0.5f;     // scaled pivot below which the output basis is orthogonalised again

struct SvdGeom {
  int nc, nt, nw;
  int mrI, mcJ;  // rows of a row slab, columns of a column slab
  int ldr, ldc;  // leading dimensions of the slabs (floats)
  int ldy, ldx;  // column strides of the gathered blocks P|Y (nI rows) and Q|X (nJ rows), odd
  int sl, ws;    // floats per exchange slot, per warp slot
  size_t off_urow, off_ucol, off_p, off_q, off_ps, off_qs, off_red, off_w, off_small, off_r64, off_bar, total;
};

__host__ __device__ inline int svd_odd(int x) { return (x & 1) ? x : x + 1; }

__host__ __device__ inline SvdGeom svd_geom(int nI, int nJ, int R, int nc) {
  SvdGeom g;
  g.nc = nc;
  g.nt = nc == 1 ? kSvdThreadsOne : kSvdThreadsCl;
  g.nw = g.nt / 32;
  // cluster form: row slabs of a multiple of 4 rows, so that the transposed
  // quads each CTA pushes into the column slabs start on 16-byte boundaries
  g.mrI = nc == 1 ? nI : (((nI + nc - 1) / nc + 3) & ~3);
  g.mcJ = (nJ + nc - 1) / nc;
  // NC = 1: one copy of the core, odd row stride (rows and columns conflict-free);
  // NC > 1: 16-byte rows (bulk copies), any stride is conflict-free for the lanes-over-k reads
  g.ldr = nc == 1 ? svd_odd(nJ) : ((nJ + 3) & ~3);
  g.ldc = (nI + 3) & ~3;  // 16-byte rows: the pushed quads are 16-byte stores
  g.ldy = svd_odd(nI);
  g.ldx = svd_odd(nJ);
  g.sl = svd_slot(R);
  g.ws = svd_wslot(R);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return o;
  };
  g.off_urow = take((size_t)(nc == 1 ? nI : g.mrI) * g.ldr * 4);
  g.off_ucol = take(nc == 1 ? 0 : (size_t)g.mcJ * g.ldc * 4);
  g.off_p = take((size_t)R * g.ldy * 4);
  g.off_q = take((size_t)R * g.ldx * 4);
  g.off_ps = take((size_t)nc * g.sl * 4);
  g.off_qs = take((size_t)nc * g.sl * 4);
  g.off_red = take((size_t)g.nw * g.sl * 4);
  g.off_w = take((size_t)(svd_rep(R) ? g.nw : 1) * g.ws * 4);
  g.off_small = take((size_t)(3 * R * R + R + 16) * 4);
  g.off_r64 = take((size_t)(g.nt + svd_np(R)) * 8);
  g.off_bar = take(16);
  g.total = off;
  return g;
}

// ---------------------------------------------------------------------------
// warp building blocks

// Reduce-scatter of NV (a power of two <= 32) values across the warp: lane L
// returns the sum over all 32 lanes of element L % NV (a fixed summation order).
template <int NV>
__device__ __forceinline__ float warp_rs(float (&v)[NV]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = NV / 2; h >= 1; h >>= 1) {
    const bool hi = (lane & h) != 0;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = hi ? v[j] : v[j + h];
      const float keep = hi ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  float x = v[0];
#pragma unroll
  for (int o = NV; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int R>
__device__ __forceinline__ void pair_of(int p, int& s, int& t) {
  s = 0;
  int rem = p;
  while (rem >= R - s) {
    rem -= R - s;
    ++s;
  }
  t = s + rem;
}

template <int R>
__device__ __forceinline__ float selr(const float (&g)[R], int t) {
  float v = 0.f;
#pragma unroll
  for (int u = 0; u < R; ++u)
    if (u == t) v = g[u];
  return v;
}

// One slab product for a group of G <= svd_gmax(R) output rows starting at
// `row0`: out(row, t) = sum over the inner index k < ninner of
// base[row * rs + k * ks] * M[t * ldm + k].  Lanes run over k; the G R partial
// sums are reduce-scattered, so lane L < G R returns out(row0 + L / R, L % R).
// Rows >= nvalid contribute zero.
template <int R>
__device__ __forceinline__ float slab_product(const float* __restrict__ base, int rs, int ks, int row0, int G,
                                              int nvalid, int ninner, const float* __restrict__ M, int ldm) {
  constexpr int GM = svd_gmax(R);
  constexpr int NV = svd_pow2(GM * R);
  const int lane = threadIdx.x & 31;
  float v[NV];  // v[g R + t]: partial sum of out(row0 + g, t)
#pragma unroll
  for (int e = 0; e < NV; ++e) v[e] = 0.f;
#pragma unroll 2
  for (int k = lane; k < ninner; k += 32) {
    float mv[R];
#pragma unroll
    for (int t = 0; t < R; ++t) mv[t] = M[t * ldm + k];
    const float* up = base + (size_t)k * ks + (size_t)row0 * rs;
#pragma unroll
    for (int g = 0; g < GM; ++g) {
      if (g < G && row0 + g < nvalid) {
        const float u = up[(size_t)g * rs];
#pragma unroll
        for (int t = 0; t < R; ++t) v[g * R + t] = fmaf(u, mv[t], v[g * R + t]);
      }
    }
  }
  return warp_rs<NV>(v);
}

// Accumulate the Gram pairs of a group's rows from their reduce-scattered
// values (lane g R + t holds row g, column t): gp[q] += sum_g v(g,s) v(g,t) for
// the pairs p = lane + 32 q (upper triangle, row-major pair order).
template <int R>
__device__ __forceinline__ void group_gram(float val, int G, const int (&ps)[(svd_np(R) + 31) / 32],
                                           const int (&pt)[(svd_np(R) + 31) / 32],
                                           float (&gp)[(svd_np(R) + 31) / 32]) {
  constexpr int GM = svd_gmax(R);
  constexpr int PQ = (svd_np(R) + 31) / 32;
#pragma unroll
  for (int g = 0; g < GM; ++g) {
    if (g < G) {
#pragma unroll
      for (int q = 0; q < PQ; ++q) {
        const float a = __shfl_sync(0xffffffffu, val, g * R + ps[q]);
        const float b = __shfl_sync(0xffffffffu, val, g * R + pt[q]);
        gp[q] = fmaf(a, b, gp[q]);
      }
    }
  }
}

// Cholesky factor of the R x R Gram matrix G (full, row-major, in shared
// memory) formed by one warp in registers (lane l holds row l of the Schur
// complement): G = U^T U, U upper triangular written to Uw (U(t,u) at t R + u),
// reciprocal pivots to dw.  Pivots <= 1e-12 of the largest diagonal entry mark
// dependent columns (zero rows of U, dw = 0).  Returns the number of those and,
// in minsp, the smallest pivot above noise level relative to its column's
// diagonal entry of G (1 for an orthogonal block; small values mean FP32
// cancellation).
template <int R>
__device__ int warp_chol(const float* G, int r, float* Uw, float* dw, float& minsp) {
  const int lane = threadIdx.x & 31;
  float g[R];
#pragma unroll
  for (int u = 0; u < R; ++u) g[u] = (lane < r && u < r) ? G[lane * R + u] : 0.f;
  const float gdiag = selr<R>(g, lane);
  float maxd = gdiag;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxd = fmaxf(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
  int brk = 0;
  float msp = 1.f;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    if (t < r) {  // the same in every lane
      const float dgt = __shfl_sync(0xffffffffu, g[t], t);
      const float g0t = __shfl_sync(0xffffffffu, gdiag, t);
      const bool keep = dgt > 1e-12f * maxd && dgt <= FLT_MAX;
      const float rinv = keep ? rsqrtf(dgt) : 0.f;
      // a column whose own diagonal entry is below 1e-10 of the largest is FP32
      // noise of the products themselves (sigma_t / sigma_1 < 1e-5, below the
      // FP32 rank cutoff): FP64 could not recover it, so it does not count.  A
      // live column whose pivot collapsed (small, zero or negative: FP32
      // cancellation in an ill-conditioned block) reads as 0 and calls for the
      // FP64 factor.
      if (g0t > 1e-10f * maxd) msp = fminf(msp, keep ? __fdividef(dgt, g0t) : 0.f);
      const float ul = g[t] * rinv;  // U(t, lane)
      float urow[R];
#pragma unroll
      for (int u = 0; u < R; ++u) urow[u] = __shfl_sync(0xffffffffu, ul, u);
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < R; ++u) Uw[t * R + u] = (u >= t) ? urow[u] : 0.f;
        dw[t] = rinv;
      }
      if (lane > t) {
#pragma unroll
        for (int u = t + 1; u < R; ++u) g[u] = fmaf(-ul, urow[u], g[u]);
      }
      brk += keep ? 0 : 1;
    } else if (lane == 0) {
      dw[t] = 0.f;
#pragma unroll
      for (int u = 0; u < R; ++u) Uw[t * R + u] = 0.f;
    }
  }
  __syncwarp();
  minsp = msp;
  return brk;
}

// Cholesky factor of the R x R Gram matrix G (full, row-major, shared memory)
// formed in every lane's registers, with the FMA order of warp_chol (so the
// same factor bit for bit): no shuffles on the dependent path.
template <int R>
__device__ int lane_chol(const float* G, int r, float* Uw, float* dw, float& minsp) {
  const int lane = threadIdx.x & 31;
  float a[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) a[i][j] = (i < r && j < r && j >= i) ? G[i * R + j] : 0.f;
  float maxd = 0.f;
#pragma unroll
  for (int i = 0; i < R; ++i) maxd = fmaxf(maxd, a[i][i]);
  float g0[R];
#pragma unroll
  for (int i = 0; i < R; ++i) g0[i] = a[i][i];
  int brk = 0;
  float msp = 1.f;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    if (t < r) {
      const float dgt = a[t][t];
      const bool keep = dgt > 1e-12f * maxd && dgt <= FLT_MAX;
      const float rinv = keep ? rsqrtf(dgt) : 0.f;
      if (g0[t] > 1e-10f * maxd) msp = fminf(msp, keep ? __fdividef(dgt, g0[t]) : 0.f);
      float urow[R];
#pragma unroll
      for (int u = 0; u < R; ++u) urow[u] = (u >= t) ? a[t][u] * rinv : 0.f;
      if (lane == 0) {
#pragma unroll
        for (int u = 0; u < R; ++u) Uw[t * R + u] = urow[u];
        dw[t] = rinv;
      }
#pragma unroll
      for (int i = t + 1; i < R; ++i)
#pragma unroll
        for (int u = i; u < R; ++u) a[i][u] = fmaf(-urow[i], urow[u], a[i][u]);
      brk += keep ? 0 : 1;
    } else if (lane == 0) {
      dw[t] = 0.f;
#pragma unroll
      for (int u = 0; u < R; ++u) Uw[t * R + u] = 0.f;
    }
  }
  __syncwarp();
  minsp = msp;
  return brk;
}

// The same factorisation in FP64 from an FP64 Gram matrix (pairs, upper
// triangle); the factor and reciprocal pivots are stored in FP32.
template <int R>
__device__ void warp_chol64(const double* Gp, int r, float* Uw, float* dw) {
  const int lane = threadIdx.x & 31;
  double g[R];
#pragma unroll
  for (int u = 0; u < R; ++u) {
    const int s = lane < u ? lane : u, t = lane < u ? u : lane;
    g[u] = (lane < r && u < r) ? Gp[s * R - s * (s - 1) / 2 + (t - s)] : 0.0;
  }
  double maxd = 0.0;
#pragma unroll
  for (int u = 0; u < R; ++u)
    if (u == lane) maxd = g[u];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxd = fmax(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
  for (int t = 0; t < r; ++t) {
    double gt = 0.0;
#pragma unroll
    for (int u = 0; u < R; ++u)
      if (u == t) gt = g[u];
    const double dgt = __shfl_sync(0xffffffffu, gt, t);
    const bool keep = dgt > 1e-24 * maxd;
    const double rs = keep ? 1.0 / sqrt(dgt) : 0.0;
    const double ul = gt * rs;
    double urow[R];
#pragma unroll
    for (int u = 0; u < R; ++u) urow[u] = __shfl_sync(0xffffffffu, ul, u);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < R; ++u) Uw[t * R + u] = (u >= t) ? (float)urow[u] : 0.f;
      dw[t] = (float)rs;
    }
    if (lane > t) {
#pragma unroll
      for (int u = 0; u < R; ++u) g[u] = fma(-ul, urow[u], g[u]);
    }
  }
  if (lane == 0) {
    for (int t = r; t < R; ++t) {
      dw[t] = 0.f;
      for (int u = 0; u < R; ++u) Uw[t * R + u] = 0.f;
    }
  }
  __syncwarp();
}

// y U = m for one row (forward substitution with U from warp_chol).
template <int R>
__device__ __forceinline__ void row_subst(const float (&m)[R], float (&y)[R], const float* Uw, const float* dw) {
#pragma unroll
  for (int t = 0; t < R; ++t) {
    float v = m[t];
#pragma unroll
    for (int s2 = 0; s2 < t; ++s2) v = fmaf(-y[s2], Uw[s2 * R + t], v);
    y[t] = v * dw[t];
  }
}

// Rows i < n of a column-major block (entry (i,t) at t ld + i) replaced by
// their solutions y U = row (whole block, one row per thread).
template <int R>
__device__ __forceinline__ void block_subst(float* M, int ld, int n, const float* Uw, const float* dw) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float m[R], y[R];
#pragma unroll
    for (int t = 0; t < R; ++t) m[t] = M[t * ld + i];
    row_subst<R>(m, y, Uw, dw);
#pragma unroll
    for (int t = 0; t < R; ++t) M[t * ld + i] = y[t];
  }
}

// Rows i < n of a column-major block replaced by row * Z (Z R x R row-major).
template <int R>
__device__ __forceinline__ void block_rotate(float* M, int ld, int n, const float* Z) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float m[R];
#pragma unroll
    for (int t = 0; t < R; ++t) m[t] = M[t * ld + i];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float v = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) v = fmaf(m[s2], Z[s2 * R + t], v);
      M[t * ld + i] = v;
    }
  }
}

// Gram pairs of a whole column-major block (rows < n), FP32 or FP64, by all
// threads: thread q takes pair q % NP over the rows of chunk q / NP; the chunk
// sums are added in chunk order.  Result in gout[p] (shared, NP values).
template <int R, typename A>
__device__ void block_gram(const float* M, int ld, int n, A* scratch, A* gout) {
  constexpr int NP = svd_np(R);
  const int nch = (int)blockDim.x / NP;
  const int q = threadIdx.x;
  if (q < nch * NP) {
    const int p = q % NP, c = q / NP;
    int s, t;
    pair_of<R>(p, s, t);
    A acc = 0;
    for (int i = c; i < n; i += nch) acc += (A)M[s * ld + i] * (A)M[t * ld + i];
    scratch[c * NP + p] = acc;
  }
  __syncthreads();
  if (q < NP) {
    A acc = 0;
    for (int c = 0; c < nch; ++c) acc += scratch[c * NP + q];
    gout[q] = acc;
  }
  __syncthreads();
}

// Expand Gram pairs (upper triangle) to a full symmetric R x R matrix (one warp).
template <int R>
__device__ __forceinline__ void warp_expand(const float* gp, float* G) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < R * R; e += 32) {
    const int i = e / R, j = e - i * R;
    const int s = i < j ? i : j, t = i < j ? j : i;
    G[e] = gp[s * R - s * (s - 1) / 2 + (t - s)];
  }
  __syncwarp();
}

// Round-robin (circle method) partner of player p in round k of n (even) players.
__device__ __forceinline__ int rr_partner(int p, int k, int n) {
  if (p == n - 1) return k;
  if (p == k) return n - 1;
  int q = (2 * k - p) % (n - 1);
  return q < 0 ? q + n - 1 : q;
}

// One-sided Jacobi SVD of the r x r matrix T (T(i,p) at i R + p) in one warp,
// lane p owning column p: T Vt = Ut diag(sg), written sorted by descending
// singular value (ties: smaller column first) to Ut, Vt (row-major R x R) and
// sg; entries beyond r are zero.  A sweep rotates every column pair whose
// inner product exceeds 1e-6 of its norms (FP32 rounding of the products sits
// just below); at most 10 sweeps.
template <int R>
__device__ void warp_jacobi(const float* T, int r, float* Ut, float* Vt, float* sg) {
  const int p = threadIdx.x & 31;
  float tc[R], vc[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    tc[i] = (p < r && i < r) ? T[i * R + p] : 0.f;
    vc[i] = (i == p && p < r) ? 1.f : 0.f;
  }
  const int nplay = (r + 1) & ~1;
  for (int sweep = 0; sweep < 10; ++sweep) {
    int rotated = 0;
    for (int rnd = 0; rnd < nplay - 1; ++rnd) {
      const int q = (p < nplay) ? rr_partner(p, rnd, nplay) : p;
      float tq[R], vq[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        tq[i] = __shfl_sync(0xffffffffu, tc[i], q);
        vq[i] = __shfl_sync(0xffffffffu, vc[i], q);
      }
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
            const float va = lo ? vc[i] : vq[i], vb = lo ? vq[i] : vc[i];
            vc[i] = lo ? (c * va - s * vb) : (s * va + c * vb);
          }
        }
      }
    }
    if (!__any_sync(0xffffffffu, rotated)) break;
  }
  float s2 = 0.f;
#pragma unroll
  for (int i = 0; i < R; ++i) s2 = fmaf(tc[i], tc[i], s2);
  const float sv = (p < r) ? sqrtf(s2) : -1.f;
  int pos = 0;
  for (int q = 0; q < r; ++q) {
    const float sq = __shfl_sync(0xffffffffu, sv, q);
    pos += (sq > sv) || (sq == sv && q < p);
  }
  if (p < r) {
    const float inv = sv > 0.f ? 1.f / sv : 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      Ut[i * R + pos] = tc[i] * inv;
      Vt[i * R + pos] = vc[i];
    }
    sg[pos] = sv;
  }
  if (p == 0) {
    for (int c = r; c < R; ++c) {
      sg[c] = 0.f;
      for (int i = 0; i < R; ++i) {
        Ut[i * R + c] = 0.f;
        Vt[i * R + c] = 0.f;
      }
    }
    for (int i = r; i < R; ++i)
      for (int c = 0; c < r; ++c) {
        Ut[i * R + c] = 0.f;
        Vt[i * R + c] = 0.f;
      }
  }
  __syncwarp();
}

__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t ctr) {
  const uint64_t h = splitmix64(seed ^ splitmix64(ctr));
  return (float)(h >> 40) * (1.0f / 16777216.0f) * 2.0f - 1.0f;
}

// A random start for the subspace iteration (first iteration, B_0 = 0, or a
// warm start that lost rank): r columns of uniform [-1, 1) entries from a
// counter-based hash of (seed, k, entry), zero columns beyond r.
template <int R>
__device__ __forceinline__ void svd_random_start(float* Q, int ldx, int nJ, int r, uint64_t seed, int k) {
  for (int q = threadIdx.x; q < nJ * R; q += blockDim.x) {
    const int t = q / nJ, b = q - t * nJ;
    Q[t * ldx + b] = (t < r) ? hash_uniform(seed ^ 0x5bd1e995ull, ((uint64_t)k << 32) ^ (uint64_t)(b * R + t)) : 0.f;
  }
}

// ---------------------------------------------------------------------------
// The kernel body.  role 0: the core and its truncation on a cluster of NC
// CTAs.  Roles 1, 2 (IRCUR-R with its own sampler): rank 0 of that cluster
// draws the next iteration's I (role 1) or J (role 2) while role 0 runs.

struct SvdPtrs {
  float* urow;
  float* ucol;
  float* P;  // gathered P, then Y (column-major, nI rows)
  float* Q;  // gathered Q, then X (column-major, nJ rows)
  float* ps;
  float* qs;
  float* red;
  float* wbase;
  float* T;
  float* Ut;
  float* Vt;
  float* sg;
  int* ib;
  double* r64;
  uint64_t* bar;
};

__device__ __forceinline__ SvdPtrs svd_ptrs(unsigned char* smem, const SvdGeom& g, int R) {
  SvdPtrs p;
  p.urow = reinterpret_cast<float*>(smem + g.off_urow);
  p.ucol = reinterpret_cast<float*>(smem + g.off_ucol);
  p.P = reinterpret_cast<float*>(smem + g.off_p);
  p.Q = reinterpret_cast<float*>(smem + g.off_q);
  p.ps = reinterpret_cast<float*>(smem + g.off_ps);
  p.qs = reinterpret_cast<float*>(smem + g.off_qs);
  p.red = reinterpret_cast<float*>(smem + g.off_red);
  p.wbase = reinterpret_cast<float*>(smem + g.off_w);
  p.T = reinterpret_cast<float*>(smem + g.off_small);
  p.Ut = p.T + R * R;
  p.Vt = p.Ut + R * R;
  p.sg = p.Vt + R * R;
  p.ib = reinterpret_cast<int*>(p.sg + R);
  p.r64 = reinterpret_cast<double*>(smem + g.off_r64);
  p.bar = reinterpret_cast<uint64_t*>(smem + g.off_bar);
  return p;
}

__device__ __forceinline__ void svd_barrier(cg::cluster_group& cl, int nc) {
  if (nc > 1)
    cl.sync();
  else
    __syncthreads();
}

// Gram matrix of the exchange slots (summed in cluster-rank order) into the
// warp's G, the residual sum and the agreement flag; then the warp's Cholesky
// factor.  Every warp (or warp 0 only, without replicated factors) runs it.
template <int R>
__device__ __forceinline__ int svd_factor(const float* slots, int nc, int sl, int r, float* Gw, float* F, float* dF,
                                          float& e2, int& bad, float& minsp, float& trace) {
  constexpr int NP = svd_np(R);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int e0 = 0; e0 < R * R; e0 += 32) {
    const int e = e0 + lane;
    if (e < R * R) {
      const int i = e / R, j = e - i * R;
      const int s = i < j ? i : j, t = i < j ? j : i;
      const int p = s * R - s * (s - 1) / 2 + (t - s);
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < kSvdMaxNC; ++c)
        if (c < nc) acc += slots[c * sl + p];  // rank order
      Gw[e] = acc;
    }
  }
  float ee = 0.f, bb = 0.f;
#pragma unroll
  for (int c = 0; c < kSvdMaxNC; ++c) {
    if (c < nc) {
      ee += slots[c * sl + NP];
      bb = fmaxf(bb, slots[c * sl + NP + 1]);
    }
  }
  e2 = ee;
  bad = bb != 0.f;
  __syncwarp();
  float tr = 0.f;
#pragma unroll
  for (int t = 0; t < R; ++t) tr += t < r ? Gw[t * R + t] : 0.f;
  trace = tr;
  // up to R = 8 the whole factor fits a lane's registers (no shuffles)
  if constexpr (R <= 8)
    return lane_chol<R>(Gw, r, F, dF, minsp);
  else
    return warp_chol<R>(Gw, r, F, dF, minsp);
}

// IRCUR-R: the index sets of iteration k + 2 on one axis (0: I, 1: J) and
// their map (the panel pass of iteration k + 1 reads them before it waits for
// its core SVD); drawn by the library's sampler, or only mapped when the
// caller gave them.  The drawn set is sorted, whatever the block size.
__device__ __forceinline__ void svd_sample_ahead(const IterDesc& d, int k, int axis, SamplerSmem& S) {
  const int dn = k + 2;
  if (!d.resample || dn >= d.max_iter) return;
  const int m = axis ? d.nJ : d.nI;
  int* out = const_cast<int*>(axis ? d.J_all : d.I_all) + (int64_t)dn * m;
  unsigned* map = axis ? d.posJ[dn & 1] : d.posI[dn & 1];
  if (d.sampleAhead) {
    sample_subset(d.seed, dn, axis, axis ? d.n2 : d.n1, m, out, S, map, (unsigned)(dn + 1));
  } else {
    for (int a = threadIdx.x; a < m; a += blockDim.x) map[out[a]] = index_tag((unsigned)(dn + 1), a);
  }
}

template <int R>
__device__ __forceinline__ void svd_body(const IterDesc& d, int role, unsigned char* smem, int par) {
  constexpr int NP = svd_np(R);
  constexpr int PQ = (NP + 31) / 32;
  constexpr int GM = svd_gmax(R);
  constexpr bool REP = svd_rep(R);
  constexpr int kPre = 4;  // values of this CTA's rows of A_k(I,:) a thread prefetches
  cg::cluster_group cl = cg::this_cluster();
  const int nc = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  State* st = d.st;
  // Role 0: B_k(:,J)^T, this CTA's rows of A_k(I,:) and T's diagonal from the
  // buffers of this launch's parity, loaded before the state (their latency
  // overlaps its load); reloaded below in the (unexpected) case that the
  // parity differs from k's.
  const SvdGeom g0 = svd_geom(d.nI, d.nJ, R, nc);
  const int prow0 = nc == 1 ? 0 : crank * g0.mrI;
  const int pnrw = nc == 1 ? d.nI : (d.nI - prow0 < g0.mrI ? (d.nI - prow0 > 0 ? d.nI - prow0 : 0) : g0.mrI);
  const int pq0 = threadIdx.x, pq1 = threadIdx.x + (int)blockDim.x;
  float bj0[R], bj1[R], tdiag[R], apre[kPre];
  const bool pre_ai = pnrw * R <= kPre * (int)blockDim.x;
  auto load_side = [&](int pb) {
    const float* BJp = d.BJt[pb];
    const float* AIp = d.AI[pb];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      bj0[t] = pq0 < d.nJ ? BJp[(size_t)pq0 * R + t] : 0.f;
      bj1[t] = pq1 < d.nJ ? BJp[(size_t)pq1 * R + t] : 0.f;
      tdiag[t] = d.Tm[t * R + t];
    }
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      const int q = (int)threadIdx.x + u * (int)blockDim.x;
      apre[u] = (pre_ai && q < pnrw * R) ? AIp[(size_t)prow0 * R + q] : 0.f;
    }
  };
  if (role == 0) load_side(par & 1);
  if (st->done || st->status) return;  // the same for every CTA: the state is fixed during the launch
  const int k = st->k;
  if (role == 0 && (k & 1) != (par & 1)) load_side(k & 1);
  if (role > 0) {
    if (crank == 0) svd_sample_ahead(d, k, role - 1, *reinterpret_cast<SamplerSmem*>(smem));
    return;
  }
  if (crank == 0) {
    trace_start(d.trace, kTraceSlots * k + 0);
    trace_start(d.trace, kTraceSlots * k + 1);
  }
  const int nI = d.nI, nJ = d.nJ, r = d.r;
  const SvdGeom g = svd_geom(nI, nJ, R, nc);
  const SvdPtrs sp = svd_ptrs(smem, g, R);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NW = (int)(blockDim.x >> 5);
  const int row0 = nc == 1 ? 0 : crank * g.mrI;
  const int nrw = nc == 1 ? nI : (nI - row0 < g.mrI ? (nI - row0 > 0 ? nI - row0 : 0) : g.mrI);
  const int col0 = nc == 1 ? 0 : crank * g.mcJ;
  const int ncl = nc == 1 ? nJ : (nJ - col0 < g.mcJ ? (nJ - col0 > 0 ? nJ - col0 : 0) : g.mcJ);
  float* Wsl = sp.wbase + (REP ? (size_t)warp * g.ws : 0);
  float* Gw = Wsl;
  float* F1 = Gw + R * R;
  float* d1 = F1 + R * R;
  float* F2 = d1 + R;
  float* d2 = F2 + R * R;
  const float zeta = (float)st->zeta;
  const float* AIk = d.AI[k & 1];   // A_k(I_k,:), nI x R
  const int buf = d.resample ? (k & 1) : 0;
  const float* Dc = d.Dc[buf];

  // ---- 1. bulk copies of this CTA's rows of D(I,J) (cluster form)
  const bool bulk = nc > 1;
  if (bulk && warp == 0) {
    const unsigned rowb = (unsigned)(((nJ + 3) & ~3) * 4);
    if (lane == 0) {
      mbar_init(sp.bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(sp.bar, (unsigned)nrw * rowb);
    }
    __syncwarp();
    for (int i = lane; i < nrw; i += 32) bulk_g2s(sp.urow + (size_t)i * g.ldr, Dc + (size_t)(row0 + i) * d.ldDc, rowb, sp.bar);
  }
  // ---- 2. this CTA's rows of A_k(I,:) to its own rows of P (rows of P owned
  // by other CTAs may already hold their first pushed product: nothing orders
  // another CTA's first half-step after this prologue, but this CTA's own rows
  // are written by this CTA alone), and B_k(:,J)^T in registers (thread q:
  // rows q and q + blockDim), both compact copies the previous panel pass wrote.
  // The warm start X_0 = B_k(:,J)^T diag(1 / |T_tt|), T the previous core's
  // (H_r = Y T X^T, T near-diagonal in the graded basis): B_k(:,J)^T is close
  // to X' T^T, so the scaling leaves columns of comparable norm, as the
  // dependence cutoff of the Cholesky factor (relative to its largest diagonal
  // entry) assumes.  k = 0 (B_0 = 0): a random start.
  const int q0 = tid, q1 = tid + (int)blockDim.x;
  {
    float inv[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const float tt = (k > 0 && t < r) ? fabsf(tdiag[t]) : 0.f;
      inv[t] = tt > 0.f ? 1.f / tt : 0.f;
    }
    if (pre_ai) {
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        const int q = tid + u * (int)blockDim.x;
        if (q < nrw * R) {
          const int il = q / R, t = q - il * R;
          sp.P[t * g.ldy + row0 + il] = apre[u];
        }
      }
    } else {
      for (int q = tid; q < nrw * R; q += blockDim.x) {
        const int il = q / R, t = q - il * R;
        sp.P[t * g.ldy + row0 + il] = AIk[(size_t)(row0 + il) * R + t];
      }
    }
    if (k > 0) {
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (q0 < nJ) sp.Q[t * g.ldx + q0] = bj0[t] * inv[t];
        if (q1 < nJ) sp.Q[t * g.ldx + q1] = bj1[t] * inv[t];
      }
    } else {
      svd_random_start<R>(sp.Q, g.ldx, nJ, r, d.seed, k);
    }
  }
  __syncthreads();
  // ---- 3. Phase I on the core, this CTA's rows:
  // D(I,J) - T_zeta(D(I,J) - L_k(I,J)).  Each entry is formed once, in the row
  // slab, which is then pushed to the CTAs that own its columns (column slabs,
  // stored transposed); the first half-step's cluster barrier publishes those
  // pushes before any CTA's first product with the column slab.
  bool ok = true;
  if (bulk) {
    ok = mbar_wait_bounded(sp.bar, 0, d.spinLimit);
    if (!ok) {
      if (tid == 0) atomicExch(&st->status, (int)IRCUR_ETIMEOUT);
      mbar_wait_bounded(sp.bar, 0, kSpinLimit);  // let the copy land before the block exits
    }
    ok = __syncthreads_and(ok);
  }
  {
    // one entry: D - S with S = T_zeta(D - L_k) (the BF16 variant takes the
    // panels' BF16 decision, re-taken in FP32 within the rounding band)
    auto entry = [&](float dv32, const float (&a)[R], const float (&b)[R]) {
      const float l = lowrank_entry<R>(a, b);
      const float dv = d.bf16 ? bf16_entry(f32_to_bf16_bits(dv32), l, zeta, [&]() { return dv32; }) : dv32;
      return panel_value(dv, l, zeta);
    };
    // thread per column (B_k(:,J_j) in registers), the rows' A_k(I_i,:)
    // broadcast reads of own rows of P.  The one-CTA form, whose threads
    // outnumber the columns, gives each column to ngrp threads, each with a
    // share of the rows (the first group holds B_k(:,J_j) already, the others
    // read it from the compact copy).
    const int ngrp = (nc == 1 && nJ > 0 && (int)blockDim.x >= 2 * nJ) ? (int)blockDim.x / nJ : 1;
    for (int half = 0; half < 2; ++half) {
      int j, ra = 0, rb = nrw;
      float bj[R];
      if (ngrp > 1) {
        const int grp = tid / nJ;
        if (half == 1 || grp >= ngrp) continue;
        j = tid - grp * nJ;
        ra = grp * nrw / ngrp;
        rb = (grp + 1) * nrw / ngrp;
        const float* BJc = d.BJt[k & 1];
#pragma unroll
        for (int t = 0; t < R; ++t) bj[t] = grp == 0 ? bj0[t] : BJc[(size_t)j * R + t];
      } else {
        j = half ? q1 : q0;
        if (j >= nJ) continue;
#pragma unroll
        for (int t = 0; t < R; ++t) bj[t] = half ? bj1[t] : bj0[t];
      }
      int il = ra;
      for (; il + 4 <= rb; il += 4) {
        float a4[4][R], d4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = row0 + il + u;
#pragma unroll
          for (int t = 0; t < R; ++t) a4[u][t] = sp.P[t * g.ldy + i];
          d4[u] = bulk ? sp.urow[(size_t)(il + u) * g.ldr + j] : __ldg(Dc + (size_t)i * d.ldDc + j);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          sp.urow[(size_t)(il + u) * g.ldr + j] = entry(d4[u], a4[u], bj);
        }
      }
      for (; il < rb; ++il) {
        const int i = row0 + il;
        float a1[R];
#pragma unroll
        for (int t = 0; t < R; ++t) a1[t] = sp.P[t * g.ldy + i];
        const float dv = bulk ? sp.urow[(size_t)il * g.ldr + j] : __ldg(Dc + (size_t)i * d.ldDc + j);
        sp.urow[(size_t)il * g.ldr + j] = entry(dv, a1, bj);
      }
    }
  }
  __syncthreads();
  if (nc > 1) {
    // the row slab to the column slabs, transposed: quads of four consecutive
    // rows of one column (16-byte stores; rows past the core read as zero)
    const int nq = (nrw + 3) >> 2;
    for (int q = tid; q < nq * nJ; q += blockDim.x) {
      const int j = q / nq, quad = q - j * nq, il = 4 * quad;
      float4 v;
      v.x = il + 0 < nrw ? sp.urow[(size_t)(il + 0) * g.ldr + j] : 0.f;
      v.y = il + 1 < nrw ? sp.urow[(size_t)(il + 1) * g.ldr + j] : 0.f;
      v.z = il + 2 < nrw ? sp.urow[(size_t)(il + 2) * g.ldr + j] : 0.f;
      v.w = il + 3 < nrw ? sp.urow[(size_t)(il + 3) * g.ldr + j] : 0.f;
      const int owner = j / g.mcJ;
      float* loc = sp.ucol + (size_t)(j - owner * g.mcJ) * g.ldc + row0 + il;
      float* dst = owner == crank ? loc : cl.map_shared_rank(loc, owner);
      *reinterpret_cast<float4*>(dst) = v;
    }
  }
  if (crank == 0) trace_stop(d.trace, kTraceSlots * d.max_iter, kTraceSlots * k + 0);
  float msp;

  // ---- 4. half-steps
  int ps_[PQ], pt_[PQ];
#pragma unroll
  for (int q = 0; q < PQ; ++q) {
    const int p = lane + 32 * q;
    int s = 0, t = 0;
    if (p < NP) pair_of<R>(p, s, t);
    ps_[q] = s;
    pt_[q] = t;
  }
  const int rowsP = nrw, rowsQ = ncl;
  int Gp = (rowsP + NW - 1) / NW;
  Gp = Gp < 1 ? 1 : (Gp > GM ? GM : Gp);
  int Gq = (rowsQ + NW - 1) / NW;
  Gq = Gq < 1 ? 1 : (Gq > GM ? GM : Gq);
  const float* qbase = nc > 1 ? sp.ucol : sp.urow;
  const int qrs = nc > 1 ? g.ldc : 1, qks = nc > 1 ? 1 : g.ldr;
  int h = 0;
  int exit_kind = 0;  // 1: after a P half-step (T = Rp), 2: after a Q half-step (T = Uq^T)
  unsigned flags = 0u;
  float prev_res = -1.f, prev2_res = -1.f, nrmP = 0.f;
  float rho1 = 1.f, rho2 = 1.f;  // contraction ratios of the two previous tests
  const float floor_rel = 0.5f * (0.5f * FLT_EPSILON) * sqrtf((float)(nI > nJ ? nI : nJ));
  float mspP = 1.f, mspQ = 1.f;
  bool susY = false, susX = false;
  bool abort_all = false;
  bool restarted = k == 0;  // k = 0 starts at random already
  const int maxh = 2 * d.svdMaxSteps;
  while (true) {
    const bool isP = (h & 1) == 0;
    float* Bf = isP ? sp.P : sp.Q;          // block gathered this half-step
    const int ldb = isP ? g.ldy : g.ldx;
    const float* Mb = isP ? sp.Q : sp.P;    // the other side's basis (X or Y)
    const int ldm = isP ? g.ldx : g.ldy;
    const int nrows = isP ? rowsP : rowsQ;  // rows this CTA produces
    const int gbase = isP ? row0 : col0;
    const int ninner = isP ? nJ : nI;
    const int G = isP ? Gp : Gq;
    const float* Fo = isP ? F2 : F1;  // factor of the previous half-step (T of the pair it tests)
    float gp[PQ];
#pragma unroll
    for (int q = 0; q < PQ; ++q) gp[q] = 0.f;
    float eres = 0.f;
    const bool test_prev = h > 0;
    for (int grp = warp; grp * G < nrows; grp += NW) {
      const int lr0 = grp * G;
      const float val = isP ? slab_product<R>(sp.urow, g.ldr, 1, lr0, G, nrows, ninner, Mb, ldm)
                            : slab_product<R>(qbase, qrs, qks, lr0, G, nrows, ninner, Mb, ldm);
      const int gl = lane / R, tl = lane - (lane / R) * R;
      const bool mine = lane < G * R && lr0 + gl < nrows;
      const int gi = gbase + lr0 + gl;
      if (test_prev && mine) {
        // residual of the pair this product completes: own rows of the basis
        // it replaces (Y for P, X for Q) times the previous factor
        float yu = 0.f;
#pragma unroll
        for (int s2 = 0; s2 < R; ++s2) yu = fmaf(Bf[s2 * ldb + gi], Fo[tl * R + s2], yu);
        const float e = val - yu;
        eres = fmaf(e, e, eres);
      }
      __syncwarp();
      if (mine) {
#pragma unroll
        for (int c = 0; c < kSvdMaxNC; ++c) {
          if (c < nc) {
            float* dst = (c == crank) ? Bf : cl.map_shared_rank(Bf, c);
            dst[tl * ldb + gi] = val;
          }
        }
      }
      group_gram<R>(mine ? val : 0.f, G, ps_, pt_, gp);
    }
    eres = warp_sum(eres);
#pragma unroll
    for (int q = 0; q < PQ; ++q) {
      const int p = lane + 32 * q;
      if (p < NP) sp.red[warp * g.sl + p] = gp[q];
    }
    if (lane == 0) sp.red[warp * g.sl + NP] = eres;
    __syncthreads();
    float* slots = isP ? sp.ps : sp.qs;
    for (int e = tid; e < NP + 2; e += blockDim.x) {
      float s = 0.f;
      if (e <= NP) {
#pragma unroll
        for (int w = 0; w < kSvdThreadsOne / 32; ++w)
          if (w < NW) s += sp.red[w * g.sl + e];  // warp order
      } else {
        s = ok ? 0.f : 1.f;
      }
#pragma unroll
      for (int c = 0; c < kSvdMaxNC; ++c) {
        if (c < nc) {
          float* dst = (c == crank) ? slots : cl.map_shared_rank(slots, c);
          dst[crank * g.sl + e] = s;
        }
      }
    }
    svd_barrier(cl, nc);
    // ---- the factor of this half-step, in every warp
    float e2 = 0.f, minsp = 1.f, trace = 0.f;
    int bad = 0;
    float* Fn = isP ? F1 : F2;
    float* dn = isP ? d1 : d2;
    if (REP || warp == 0) svd_factor<R>(slots, nc, g.sl, r, Gw, Fn, dn, e2, bad, minsp, trace);
    if (!REP) {
      if (tid == 0) {
        sp.ib[1] = bad;
        reinterpret_cast<float*>(sp.ib)[2] = e2;
        reinterpret_cast<float*>(sp.ib)[3] = minsp;
        reinterpret_cast<float*>(sp.ib)[4] = trace;
      }
      __syncthreads();
      bad = sp.ib[1];
      e2 = reinterpret_cast<float*>(sp.ib)[2];
      minsp = reinterpret_cast<float*>(sp.ib)[3];
      trace = reinterpret_cast<float*>(sp.ib)[4];
    }
    if (bad) {
      abort_all = true;
      break;
    }
    bool fell_back = false;
    if (minsp < kPivotFp64) {
      // FP32 cancellation: the Gram matrix of the whole gathered block in FP64
      double* gout64 = sp.r64 + g.nt;
      block_gram<R, double>(Bf, ldb, isP ? nI : nJ, sp.r64, gout64);
      if (REP || warp == 0) warp_chol64<R>(gout64, r, Fn, dn);
      if (!REP) __syncthreads();
      fell_back = true;
      minsp = 0.f;
    }
    if (h == 0 && !restarted) {
      // a warm start that lost rank (a previous core of numerical rank < r)
      // leaves dependent columns in the first block (zero reciprocal pivots of
      // the final, possibly FP64, factor): the first half-step again from a
      // random start, once; a core that is itself deficient keeps its
      // dependent columns and ends with IRCUR_FLAG_WRANK
      int dep = 0;
#pragma unroll
      for (int t = 0; t < R; ++t) dep += (t < r && dn[t] == 0.f) ? 1 : 0;
      if (dep > 0) {
        restarted = true;
        __syncthreads();
        svd_random_start<R>(sp.Q, g.ldx, nJ, r, d.seed, k);
        // every CTA has summed this half-step's slots before any CTA pushes
        // the repeated half-step's
        svd_barrier(cl, nc);
        __syncthreads();
        continue;
      }
    }
    if (isP) {
      nrmP = sqrtf(trace);
      mspP = minsp;
      susY = fell_back || minsp < kRegrade;
    } else {
      mspQ = minsp;
      susX = fell_back || minsp < kRegrade;
    }
    ++h;
    // ---- convergence of the pair this half-step completed
    bool stop = false;
    if (test_prev) {
      // rho: contraction of the residual over this half-step (sigma_{r+1} /
      // sigma_r once the iteration is geometric); near the FP32 floor the
      // ratio reads ~1 whatever the gap, so the gap is judged by the best of
      // the last three ratios
      const float res = sqrtf(e2);
      const float nrm = nrmP;
      const float rho = prev_res > 0.f ? res / prev_res : 0.5f;
      const float rho_min = fminf(rho, fminf(rho1, rho2));
      const bool narrow = rho_min > 0.8f;
      const float room = fmaxf(0.05f, 1.f - fminf(rho_min, 1.f));
      // target: the truncated subspace accurate to ~1e-6 (residual / gap)
      const bool conv = res <= 1e-6f * nrm * room || !(nrm > 0.f);
      // the FP32 floor of the residual, about u sqrt(m) / 2 of ||T||
      const bool at_floor = res <= floor_rel * nrm;
      const bool stag = h >= 4 && prev2_res > 0.f && res >= 0.97f * prev2_res && res <= 1e-4f * nrm;
      if (conv || (!narrow && at_floor) || stag) stop = true;
      if (stop && !conv && narrow) flags |= IRCUR_FLAG_SVD_GAP;
      rho2 = rho1;
      rho1 = rho;
      prev2_res = prev_res;
      prev_res = res;
    }
    if (!stop && h >= maxh) {
      stop = true;
      flags |= IRCUR_FLAG_SVD_NOCONV;
    }
    // the new basis: Y = P Rp^{-1} or X = Q Uq^{-1}, in place
    block_subst<R>(Bf, ldb, isP ? nI : nJ, Fn, dn);
    if (stop) {
      exit_kind = isP ? 1 : 2;
      __syncthreads();
      break;
    }
    if (fell_back) {
      // rotate both bases to the Ritz vectors of T (= Rp, or Uq^T) so that the
      // next products are graded again; T becomes diag(sigma)
      __syncthreads();
      if (warp == 0) {
        for (int e = lane; e < R * R; e += 32) {
          const int i = e / R, j = e - i * R;
          sp.T[e] = isP ? Fn[e] : Fn[j * R + i];
        }
        __syncwarp();
        warp_jacobi<R>(sp.T, r, sp.Ut, sp.Vt, sp.sg);
      }
      __syncthreads();
      block_rotate<R>(sp.P, g.ldy, nI, sp.Ut);
      block_rotate<R>(sp.Q, g.ldx, nJ, sp.Vt);
      if (REP || warp == 0) {
        for (int e = lane; e < R * R; e += 32) {
          const int i = e / R, j = e - i * R;
          Fn[e] = (i == j) ? sp.sg[i] : 0.f;
        }
        __syncwarp();
      }
      // a faster CTA's next pushes must not land while this CTA still rotates
      svd_barrier(cl, nc);
      continue;
    }
    __syncthreads();
  }
  if (abort_all) return;  // a CTA's bulk copy timed out (ETIMEOUT is set); no remote access follows

  // ---- 5. H_r(core) = Y T X^T: orthogonality restored where the last
  // factorisations were poorly conditioned, then T = Ut Sigma Vt^T
  if (warp == 0) {
    for (int e = lane; e < R * R; e += 32) {
      const int i = e / R, j = e - i * R;
      sp.T[e] = exit_kind == 1 ? F1[e] : F2[j * R + i];
    }
  }
  __syncthreads();
  // Re-orthogonalisation Y_old = Y U2y, X_old = X U2x (Cholesky QR).  After a P
  // half-step the exact relation is core X = Y T (P = Y Rp), so
  // T <- U2y T U2x^{-1}; after a Q half-step it is Y^T core = T X^T
  // (Q = X Uq), so T <- U2y^{-T} T U2x^T.
  float* gout2 = reinterpret_cast<float*>(sp.r64 + g.nt);
  if (susY) {
    block_gram<R, float>(sp.P, g.ldy, nI, reinterpret_cast<float*>(sp.r64), gout2);
    if (warp == 0) {
      warp_expand<R>(gout2, Gw);
      warp_chol<R>(Gw, r, sp.Ut, sp.sg, msp);
      if (lane < R) {
        float col[R], z[R];
#pragma unroll
        for (int i = 0; i < R; ++i) col[i] = sp.T[i * R + lane];
        if (exit_kind == 1) {  // column of U2y T
#pragma unroll
          for (int i = 0; i < R; ++i) {
            float v = 0.f;
#pragma unroll
            for (int u = 0; u < R; ++u) v = fmaf(sp.Ut[i * R + u], col[u], v);
            z[i] = v;
          }
        } else {  // column of U2y^{-T} T: z^T U2y = col^T
          row_subst<R>(col, z, sp.Ut, sp.sg);
        }
#pragma unroll
        for (int i = 0; i < R; ++i) sp.T[i * R + lane] = z[i];
      }
    }
    __syncthreads();
    block_subst<R>(sp.P, g.ldy, nI, sp.Ut, sp.sg);
    __syncthreads();
  }
  if (susX) {
    block_gram<R, float>(sp.Q, g.ldx, nJ, reinterpret_cast<float*>(sp.r64), gout2);
    if (warp == 0) {
      warp_expand<R>(gout2, Gw);
      warp_chol<R>(Gw, r, sp.Vt, sp.sg, msp);
      if (lane < R) {
        float row[R], y[R];
#pragma unroll
        for (int t = 0; t < R; ++t) row[t] = sp.T[lane * R + t];
        if (exit_kind == 1) {  // row of T U2x^{-1}
          row_subst<R>(row, y, sp.Vt, sp.sg);
        } else {  // row of T U2x^T
#pragma unroll
          for (int j = 0; j < R; ++j) {
            float v = 0.f;
#pragma unroll
            for (int u = 0; u < R; ++u) v = fmaf(row[u], sp.Vt[j * R + u], v);
            y[j] = v;
          }
        }
#pragma unroll
        for (int t = 0; t < R; ++t) sp.T[lane * R + t] = y[t];
      }
    }
    __syncthreads();
    block_subst<R>(sp.Q, g.ldx, nJ, sp.Vt, sp.sg);
    __syncthreads();
  }
  // ---- 6. rank and outputs.  With T triangular (no re-orthogonalisation) its
  // inverse is a back substitution, and sigma_min / sigma_max >=
  // 1 / (||T||_F ||T^{-1}||_F): above the rank cutoff that certifies rank r,
  // and H_r(core) = Y T X^T with U^+ = (X T^{-1}) Y^T is output as it stands.
  // Otherwise (a possibly deficient core, a re-orthogonalised or FP64-rescued
  // basis) the Jacobi SVD T = Ut Sigma Vt^T decides the numerical rank and the
  // outputs are written in the Ritz basis.
  const float rank_tol = (float)(nI > nJ ? nI : nJ) * FLT_EPSILON;
  bool fast = !(susY || susX);
  if (warp == 0) {
    int certified = 0;
    if (fast) {
      // T upper (exit after P: Rp) or lower (after Q: Uq^T); Ut <- T^{-1}
      const float* U = exit_kind == 1 ? F1 : F2;  // upper triangular factor, rows t
      const float* du = exit_kind == 1 ? d1 : d2;
      float x[R];
      const int c = lane;
#pragma unroll
      for (int s2 = R - 1; s2 >= 0; --s2) {
        float v = (s2 == c) ? 1.f : 0.f;
#pragma unroll
        for (int u = s2 + 1; u < R; ++u) v = fmaf(-U[s2 * R + u], x[u], v);
        x[s2] = (c < r && s2 <= c) ? v * du[s2] : 0.f;
      }
      float tf = 0.f, itf = 0.f;
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) {
        if (c < R) {
          // U^{-1}(s2, c) = x[s2]; T^{-1} = U^{-1} (after P) or U^{-T} (after Q)
          if (exit_kind == 1)
            sp.Ut[s2 * R + c] = x[s2];
          else
            sp.Ut[c * R + s2] = x[s2];
        }
        itf = fmaf(x[s2], x[s2], itf);
        const float tv = c < R ? U[s2 * R + c] : 0.f;
        tf = fmaf(tv, tv, tf);
      }
      tf = warp_sum(tf);
      itf = warp_sum(itf);
      // a dropped (dependent) pivot leaves T singular: never certified
      bool allpiv = true;
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) allpiv = allpiv && (s2 >= r || du[s2] != 0.f);
      // rank r certified: 1 / (||T||_F ||T^{-1}||_F) > cutoff
      certified = (allpiv && tf > 0.f && itf > 0.f && rank_tol * rank_tol * tf * itf < 1.f && itf <= FLT_MAX) ? 1 : 0;
    }
    if (lane == 0) sp.ib[5] = certified;
  }
  __syncthreads();
  fast = fast && sp.ib[5] != 0;
  int kr = r;
  if (!fast) {
    if (warp == 0) warp_jacobi<R>(sp.T, r, sp.Ut, sp.Vt, sp.sg);
    __syncthreads();
    const float tol = rank_tol * sp.sg[0];
    kr = 0;
    for (int t = 0; t < r; ++t) kr += (sp.sg[t] > tol && sp.sg[t] > 0.f) ? 1 : 0;
  }
  {
    // one thread per output entry (row, t), this CTA's share of the rows; the
    // same FMA chain per entry as a row-per-thread loop
    const int wr = (nI + nc - 1) / nc, w0 = crank * wr, w1 = w0 + wr < nI ? w0 + wr : nI;
    for (int q = tid; q < (w1 - w0) * R; q += blockDim.x) {
      const int i = w0 + q / R, t = q - (q / R) * R;
      float v = sp.P[t * g.ldy + i];
      if (!fast) {
        v = 0.f;
#pragma unroll
        for (int s2 = 0; s2 < R; ++s2) v = fmaf(sp.P[s2 * g.ldy + i], sp.Ut[s2 * R + t], v);
      }
      d.W[(size_t)i * R + t] = t < kr ? v : 0.f;
    }
    const int vr = (nJ + nc - 1) / nc, v0 = crank * vr, v1 = v0 + vr < nJ ? v0 + vr : nJ;
    for (int q = tid; q < (v1 - v0) * R; q += blockDim.x) {
      const int j = v0 + q / R, t = q - (q / R) * R;
      float x[R];
#pragma unroll
      for (int s2 = 0; s2 < R; ++s2) x[s2] = sp.Q[s2 * g.ldx + j];
      float vs = 0.f, vv = 0.f;
      if (fast) {  // Vs = X T^{-1}, V = X T^T
#pragma unroll
        for (int s2 = 0; s2 < R; ++s2) {
          vs = fmaf(x[s2], sp.Ut[s2 * R + t], vs);
          vv = fmaf(x[s2], sp.T[t * R + s2], vv);
        }
      } else {  // Vs = X Vt Sigma^{-1}, V = X Vt Sigma
        float v = 0.f;
#pragma unroll
        for (int s2 = 0; s2 < R; ++s2) v = fmaf(x[s2], sp.Vt[s2 * R + t], v);
        vs = t < kr ? v / sp.sg[t] : 0.f;
        vv = t < kr ? v * sp.sg[t] : 0.f;
      }
      const bool kt = t < kr;
      d.Vs[(size_t)j * R + t] = kt ? vs : 0.f;
      d.V[(size_t)j * R + t] = kt ? vv : 0.f;
    }
  }
  if (crank == 0) {
    for (int e = tid; e < R * R; e += blockDim.x) {
      const int i = e / R, j = e - i * R;
      d.Tm[e] = fast ? sp.T[e] : ((i == j && i < kr) ? sp.sg[i] : 0.f);
    }
    if (tid == 0) {
      unsigned f = flags;
      if (kr < r) f |= IRCUR_FLAG_WRANK;
      if (f) atomicOr(&st->flags, f);
      st->svd_steps += h;
      st->svd_last_steps = h;
    }
    if (d.trace) {
      __syncthreads();
      trace_stop(d.trace, kTraceSlots * d.max_iter, kTraceSlots * k + 1);
    }
  }
}

// The cluster form caps its registers at 128 per thread up to R = 10, so that
// the pass blocks launched while it runs fit on its SMs.
template <int R>
__global__ void __launch_bounds__(kSvdThreadsCl, (R <= 10 ? 2 : 1)) csvd_kernel(IterDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  // every CTA is resident from here on: the pass kernel may start on the
  // other SMs (it waits for this grid before reading its outputs)
  pdl_launch_dependents();
  svd_body<R>(d, blockIdx.y, smem, d.par);
}

template <int R>
__global__ void __launch_bounds__(kSvdThreadsOne, 1) ssvd_kernel(IterDesc d) {
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_launch_dependents();
  svd_body<R>(d, blockIdx.y, smem, d.par);
}

// Batched forms: cluster (or CTA) x / NC factorises instance list[x / NC].
template <int R>
__global__ void __launch_bounds__(kSvdThreadsCl, (R <= 10 ? 2 : 1)) csvd_batch_kernel(const IterDesc* __restrict__ ds,
                                                                                    const int* __restrict__ list,
                                                                                    int par) {
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_launch_dependents();
  svd_body<R>(ds[list[blockIdx.x / cg::this_cluster().num_blocks()]], blockIdx.y, smem, par);
}

template <int R>
__global__ void __launch_bounds__(kSvdThreadsOne, 1) ssvd_batch_kernel(const IterDesc* __restrict__ ds,
                                                                      const int* __restrict__ list, int par) {
  extern __shared__ __align__(16) unsigned char smem[];
  pdl_launch_dependents();
  svd_body<R>(ds[list[blockIdx.x]], blockIdx.y, smem, par);
}

// Singular values of the last core's T (H_r(core) = Y T X^T, so they are the
// r largest singular values of H_r), on request: one warp's Jacobi SVD.
template <int R>
__global__ void sigma_kernel(const float* __restrict__ Tm, int r, float* __restrict__ sigma) {
  __shared__ float T[R * R], Ut[R * R], Vt[R * R], sg[R];
  for (int e = threadIdx.x; e < R * R; e += 32) T[e] = Tm[e];
  __syncwarp();
  warp_jacobi<R>(T, r, Ut, Vt, sg);
  if ((int)threadIdx.x < r) sigma[threadIdx.x] = sg[threadIdx.x];
}

// ---------------------------------------------------------------------------
// launches (instantiated per rank in k_svd_ranks_*.cu)

template <typename... Args>
static cudaError_t launch_svd_grid(void (*kernel)(Args...), int nc, dim3 grid, size_t smem, cudaStream_t s,
                                   Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // the largest shared-memory carveout on the SVD's SMs, so that the pass
  // blocks launched while it runs fit next to it
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess && nc > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = dim3(nc == 1 ? kSvdThreadsOne : kSvdThreadsCl, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)nc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = nc > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int R>
cudaError_t svd_launch_r(const IterDesc& d, cudaStream_t s) {
  const int nc = d.svdNC;
  const size_t bytes = svd_smem_bytes(d.nI, d.nJ, R, nc);
  const dim3 grid((unsigned)nc, d.resample ? 3 : 1, 1);
  if (nc == 1) return launch_svd_grid(ssvd_kernel<R>, 1, grid, bytes, s, d);
  return launch_svd_grid(csvd_kernel<R>, nc, grid, bytes, s, d);
}

template <int R>
cudaError_t svd_launch_batch_r(const BatchLaunch& b, cudaStream_t s) {
  for (int f = 0; f < 3; ++f) {
    const int n = b.svd_n[f];
    if (n == 0) continue;
    const int nc = f == 0 ? 1 : (f == 1 ? kSvdCluster : 16);
    const dim3 grid((unsigned)(nc * n), (unsigned)b.svd_roles, 1);
    cudaError_t e = nc == 1 ? launch_svd_grid(ssvd_batch_kernel<R>, 1, grid, b.svd_smem[f], s, b.ds, b.svd_list[f], b.par)
                            : launch_svd_grid(csvd_batch_kernel<R>, nc, grid, b.svd_smem[f], s, b.ds, b.svd_list[f], b.par);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ircur
