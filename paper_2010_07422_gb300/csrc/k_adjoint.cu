// Reverse mode of unrolled IRCUR-F: the derivative of the map D -> (L_K, S_K)
// that runs Alg. 1 with fixed index sets I, J for K iterations from L_0 = 0
// (thresholds zeta_k = gamma^k zeta_0 held fixed), applied to a cotangent
// (dL, dS).  Hard thresholding contributes its almost-everywhere derivative
// (the keep mask); the rank-r truncation its SVD perturbation derivative,
// which needs sigma_r > sigma_{r+1} of every core.
//
// Iteration k of the forward, with L_k = A_k B_k, reads D and L_k only on the
// panels:  R = mix(D(I,:), L_k(I,:)), C = mix(D(:,J), L_k(:,J)),
// U~ = mix(D(I,J), L_k(I,J)) (mix = L where |D - L| > zeta_k, else D), and
// builds L_{k+1} = C H_r(U~)^+ R, which the forward holds as
// A_{k+1} = C X T^{-1}, B_{k+1} = Y^T R (H_r(U~) = Y T X^T).  A cotangent
// Gbar of L_{k+1} enters only through E = Gbar B_{k+1}^T and
// F = A_{k+1}^T Gbar, and
//     dC = E (X T^{-1})^T,   dR = Y F,
//     dP W_r = C^T E P,       (V_r^T dP)^T = R F^T P Sigma      (P = U^+),
// where T = P_T Sigma Q_T^T (an r x r SVD) gives the exact singular vectors
// W_r = Y P_T, V_r = X Q_T.  With Phi = (V_r^T dP)^T, Psi = dP W_r, the
// adjoint of U -> H_r(U)^+ is
//     Ubar = W_r G11 V_r^T + Xs V_r^T + W_r Ys^T,
//     G11 = -Sigma^{-1} (V_r^T Psi) Sigma^{-1},
//     (sigma_i^2 - M_L) Xs_i = (1 - P_W) Phi_i + Ut Psi_i / sigma_i,
//     (sigma_i^2 - M_R) Ys_i = Ut^T Phi_i / sigma_i + (1 - P_V) Psi_i,
// with Ut = (1 - P_W) U~ (1 - P_V) (the tail of U~), M_L = Ut Ut^T and
// M_R = Ut^T Ut: the derivative of the truncated SVD written as shifted
// linear systems on the complements instead of the tail's full SVD (solved by
// conjugate gradients; SPD when sigma_i > sigma_{r+1}).  The cotangent of L_k
// is the masked part of (dR, dC, Ubar) and the rest goes to dD:
//     dD(I,:) += (1 - M) dR,  dD(:,J) += (1 - M) dC,  dD(I,J) += (1 - M) Ubar,
// and its projections E_k, F_k follow from the masked parts with A_k, B_k.
// Every step is O(r |I| n2 + r |J| n1 + iters r |I| |J|): nothing dense.
#include <float.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

constexpr int kAdjThreads = 256;
constexpr int kAdjCols = 32;            // panel columns per block of the panel adjoint
constexpr int kAdjSplit = kAdjThreads / kAdjCols;  // row shares (one warp each)
constexpr int kCgThreads = 512;

// Sum of R per-thread values over the block; the result is in `out` (shared)
// for every thread after the call.
template <int R, int NT>
__device__ __forceinline__ void block_sum_R(float (&v)[R], float* red, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const float s = warp_sum(v[t]);
    if (lane == 0) red[warp * R + t] = s;
  }
  __syncthreads();
  if (threadIdx.x < R) {
    float s = 0.f;
    for (int w = 0; w < NT / 32; ++w) s += red[w * R + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}

// ---------------------------------------------------------------------------
// Final outputs: S = M_S (D - L_K), M_S = [|D - L_K| > zeta_K] (the mask of
// the reconstruction kernel, same arithmetic).  dD = M_S dS (every entry is
// written), Gbar = dL - M_S dS, E = Gbar B_K^T.  One warp per row.
template <int R>
__global__ void __launch_bounds__(kAdjThreads) adj_dense_rows_kernel(
    int64_t n1, int64_t n2, const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ D,
    int64_t ldD, const float* __restrict__ dL, int64_t lddL, const float* __restrict__ dS, int64_t lddS,
    float* __restrict__ dD, int64_t lddD, float zeta, float* __restrict__ E) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (kAdjThreads / 32) + (threadIdx.x >> 5);
  if (i >= n1) return;
  float a[R], acc[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    a[t] = A[i * R + t];
    acc[t] = 0.f;
  }
  for (int64_t j = lane; j < n2; j += 32) {
    float b[R];
#pragma unroll
    for (int t = 0; t < R; ++t) b[t] = __ldg(B + (int64_t)t * n2 + j);
    float l = 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) l = fmaf(a[t], b[t], l);
    const float d = D[i * ldD + j];
    const bool ms = fabsf(d - l) > zeta;
    const float ds = dS ? dS[i * lddS + j] : 0.f;
    const float g = (dL ? dL[i * lddL + j] : 0.f) - (ms ? ds : 0.f);
    dD[i * lddD + j] = ms ? ds : 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = fmaf(g, b[t], acc[t]);
  }
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const float s = warp_sum(acc[t]);
    if (lane == 0) E[i * R + t] = s;
  }
}

// F = A_K^T Gbar: 32 columns per block, kAdjSplit row shares, fixed-order sum.
template <int R>
__global__ void __launch_bounds__(kAdjThreads) adj_dense_cols_kernel(
    int64_t n1, int64_t n2, const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ D,
    int64_t ldD, const float* __restrict__ dL, int64_t lddL, const float* __restrict__ dS, int64_t lddS, float zeta,
    float* __restrict__ F) {
  __shared__ float red[kAdjSplit][kAdjCols][R + 1];
  const int c = threadIdx.x & 31, h = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * kAdjCols + c;
  const bool live = j < n2;
  float b[R], acc[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    b[t] = live ? B[(int64_t)t * n2 + j] : 0.f;
    acc[t] = 0.f;
  }
  const int64_t i0 = (int64_t)h * n1 / kAdjSplit, i1 = (int64_t)(h + 1) * n1 / kAdjSplit;
  if (live) {
    for (int64_t i = i0; i < i1; ++i) {
      float a[R];
#pragma unroll
      for (int t = 0; t < R; ++t) a[t] = A[i * R + t];
      float l = 0.f;
#pragma unroll
      for (int t = 0; t < R; ++t) l = fmaf(a[t], b[t], l);
      const float d = D[i * ldD + j];
      const bool ms = fabsf(d - l) > zeta;
      const float ds = dS ? dS[i * lddS + j] : 0.f;
      const float g = (dL ? dL[i * lddL + j] : 0.f) - (ms ? ds : 0.f);
#pragma unroll
      for (int t = 0; t < R; ++t) acc[t] = fmaf(a[t], g, acc[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) red[h][c][t] = acc[t];
  __syncthreads();
  if (h == 0 && live) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float s = 0.f;
      for (int hh = 0; hh < kAdjSplit; ++hh) s += red[hh][c][t];
      F[(int64_t)t * n2 + j] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Exact singular triplets of H_r(core) from the forward's Y, X T^{-1}, T:
// one-sided Jacobi on the columns of T (one warp, lane p owns column p):
// T Q = P Sigma, then W_r = Y P and V_r = X Q = (X T^{-1}) P Sigma (Q itself
// is not needed).  Order of the triplets is immaterial.
template <int R>
__global__ void __launch_bounds__(kAdjThreads) adj_small_kernel(AdjStep a) {
  __shared__ float Ps[R * R];
  __shared__ float ss[R];
  const int r = a.r;
  if (threadIdx.x < 32) {
    const int p = threadIdx.x;
    float tc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) tc[i] = (p < r && i < r) ? a.Tm[i * R + p] : 0.f;
    const int nplay = (r + 1) & ~1;
    for (int sweep = 0; sweep < 40; ++sweep) {
      int rotated = 0;
      for (int rnd = 0; rnd < nplay - 1; ++rnd) {
        // round-robin (circle method) pairing of nplay players: in round rnd
        // player nplay-1 meets rnd, and p meets 2 rnd - p (mod nplay-1)
        int q = p;
        if (p < nplay) {
          const int m = nplay - 1;
          if (p == m)
            q = rnd;
          else if (p == rnd)
            q = m;
          else
            q = (2 * rnd - p + 2 * m) % m;
        }
        float tq[R];
#pragma unroll
        for (int i = 0; i < R; ++i) tq[i] = __shfl_sync(0xffffffffu, tc[i], q);
        if (p < r && q < r && q != p) {
          const bool lo = p < q;
          float app = 0.f, aqq = 0.f, apq = 0.f;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const float x = lo ? tc[i] : tq[i];
            const float y = lo ? tq[i] : tc[i];
            app = fmaf(x, x, app);
            aqq = fmaf(y, y, aqq);
            apq = fmaf(x, y, apq);
          }
          if (fabsf(apq) > 1e-7f * sqrtf(app * aqq)) {
            rotated = 1;
            const float zz = (aqq - app) / (2.f * apq);
            const float tt = copysignf(1.f, zz) / (fabsf(zz) + sqrtf(1.f + zz * zz));
            const float cs = rsqrtf(1.f + tt * tt), sn = cs * tt;
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const float x = lo ? tc[i] : tq[i], y = lo ? tq[i] : tc[i];
              tc[i] = lo ? (cs * x - sn * y) : (sn * x + cs * y);
            }
          }
        }
      }
      if (!__any_sync(0xffffffffu, rotated)) break;
    }
    float s2 = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) s2 = fmaf(tc[i], tc[i], s2);
    const float sg = sqrtf(s2);
    if (p < R) {
      const bool ok = p < r && sg > 0.f;
      ss[p] = ok ? sg : 0.f;
#pragma unroll
      for (int i = 0; i < R; ++i) Ps[i * R + p] = ok ? tc[i] / sg : 0.f;
    }
  }
  __syncthreads();
  if (threadIdx.x < R) a.sig[threadIdx.x] = ss[threadIdx.x];
  for (int q = threadIdx.x; q < R * R; q += blockDim.x) a.Pm[q] = Ps[q];  // R * R may exceed the block
  for (int q = threadIdx.x; q < a.nI * R; q += blockDim.x) {
    const int row = q / R, p = q - row * R;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) s = fmaf(a.Y[row * R + i], Ps[i * R + p], s);
    a.Wr[q] = s;
  }
  for (int q = threadIdx.x; q < a.nJ * R; q += blockDim.x) {
    const int row = q / R, p = q - row * R;
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) s = fmaf(a.Vs[row * R + i], Ps[i * R + p], s);
    a.Vr[q] = s * ss[p];
  }
}

// ---------------------------------------------------------------------------
// Adjoint over one panel, in panel coordinates (m panel rows, 32 columns per
// block, warp h = row share h, lane = column):
//   row panel (COL = false): rows a of D(I,:), columns j;   side = A_k(I,:),
//     vec = B_k(:,j), G = F(:,j), left = Y:   dX = dR(a,j);
//   column panel (COL = true): rows b of D(:,J)^T, columns i; side = B_k(:,J)^T,
//     vec = A_k(i,:), G = E(i,:), left = X T^{-1}: dX = dC(i,b).
// Per entry: M = [|d - l| > zeta] (the forward's decision, same arithmetic),
// val = M ? l : d (the entry of R or C), gm = M dX (cotangent of L_k),
// dD += (1 - M) dX.  Per column: out = sum_a side(a,:) gm  (F_k(:,j) part f1 |
// E_k(i,:) part e2).  Per panel row, partial over the block's columns:
// [val G | gm vec] (R F^T | C^T E, and the e1 | f2 parts of E_k(I,:) | F_k(:,J)).
template <int R, bool COL>
__global__ void __launch_bounds__(kAdjThreads) adj_panel_kernel(AdjStep a) {
  extern __shared__ __align__(16) float sm[];
  const int m = COL ? a.nJ : a.nI;
  const int64_t ncolsTotal = COL ? a.n1 : a.n2;
  float* side = sm;
  float* left = side + (size_t)m * R;
  float* red = left + (size_t)m * R;  // kAdjSplit x kAdjCols x R
  for (int q = threadIdx.x; q < m * R; q += blockDim.x) {
    const int row = q / R, t = q - row * R;
    if (COL) {
      side[q] = a.Bk[(int64_t)t * a.n2 + a.J[row]];
      left[q] = a.Vs[q];
    } else {
      side[q] = a.Ak[(int64_t)a.I[row] * R + t];
      left[q] = a.Y[q];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, h = threadIdx.x >> 5;
  const int64_t j = (int64_t)blockIdx.x * kAdjCols + lane;
  const bool live = j < ncolsTotal;
  float vec[R], G[R], out[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    if (COL) {
      vec[t] = live ? a.Ak[j * R + t] : 0.f;
      G[t] = live ? a.E[j * R + t] : 0.f;
    } else {
      vec[t] = live ? a.Bk[(int64_t)t * a.n2 + j] : 0.f;
      G[t] = live ? a.F[(int64_t)t * a.n2 + j] : 0.f;
    }
    out[t] = 0.f;
  }
  const float* P = COL ? a.PcolT : a.Prow;
  const int64_t ld = COL ? a.ldPc : a.ldPr;
  float* dDp = COL ? a.dDCt : a.dDR;
  const int64_t ldd = COL ? a.n1 : a.n2;
  float* part = (COL ? a.partC : a.partR) + (size_t)blockIdx.x * m * 2 * R;
  const float zeta = a.zeta;
  const int a0 = h * m / kAdjSplit, a1 = (h + 1) * m / kAdjSplit;
  for (int row = a0; row < a1; ++row) {
    const float* sr = side + (size_t)row * R;
    const float* lf = left + (size_t)row * R;
    const float d = live ? P[(int64_t)row * ld + j] : 0.f;
    float srr[R];
#pragma unroll
    for (int t = 0; t < R; ++t) srr[t] = sr[t];
    const float l = lowrank_entry<R>(srr, vec);
    const bool msk = fabsf(d - l) > zeta;
    const float val = msk ? l : d;
    float dX = 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) dX = fmaf(lf[t], G[t], dX);
    const float gm = msk ? dX : 0.f;
    if (live && !msk) dDp[(int64_t)row * ldd + j] += dX;
#pragma unroll
    for (int t = 0; t < R; ++t) out[t] = fmaf(srr[t], gm, out[t]);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const float v1 = warp_sum(val * G[t]);
      const float v2 = warp_sum(gm * vec[t]);
      if (lane == 0) {
        part[(size_t)row * 2 * R + t] = v1;
        part[(size_t)row * 2 * R + R + t] = v2;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < R; ++t) red[((size_t)h * kAdjCols + lane) * R + t] = out[t];
  __syncthreads();
  if (h == 0 && live) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float s = 0.f;
      for (int hh = 0; hh < kAdjSplit; ++hh) s += red[((size_t)hh * kAdjCols + lane) * R + t];
      if (COL)
        a.Enew[j * R + t] = s;
      else
        a.Fnew[(int64_t)t * a.n2 + j] = s;
    }
  }
}

// Sum the per-block panel partials in block order: out1 = first R, out2 = last R.
template <int R>
__global__ void adj_reduce_kernel(const float* __restrict__ part, int tiles, int m, float* __restrict__ out1,
                                  float* __restrict__ out2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m * 2 * R) return;
  const int row = q / (2 * R), u = q - row * 2 * R;
  float s = 0.f;
  for (int tl = 0; tl < tiles; ++tl) s += part[((size_t)tl * m + row) * 2 * R + u];
  if (u < R)
    out1[row * R + u] = s;
  else
    out2[row * R + u - R] = s;
}

// The core U~ = mix(D(I,J), L_k(I,J)) into a dense nI x nJ scratch.
template <int R>
__global__ void adj_core_build_kernel(AdjStep a) {
  const int row = blockIdx.x;
  float ar[R];
#pragma unroll
  for (int t = 0; t < R; ++t) ar[t] = a.Ak[(int64_t)a.I[row] * R + t];
  for (int b = threadIdx.x; b < a.nJ; b += blockDim.x) {
    const int j = a.J[b];
    float bc[R];
#pragma unroll
    for (int t = 0; t < R; ++t) bc[t] = a.Bk[(int64_t)t * a.n2 + j];
    a.Ucore[(size_t)row * a.nJ + b] = panel_value(a.Prow[(int64_t)row * a.ldPr + j], lowrank_entry<R>(ar, bc), a.zeta);
  }
}

// ---------------------------------------------------------------------------
// Shifted systems of the truncated-SVD adjoint for one singular value
// (block i): x and y by conjugate gradients, lockstep.
struct CgSmem {
  float *W, *V, *phi, *psi, *rx, *ry, *x, *y, *px, *py, *apx, *apy, *tI, *tJ, *red, *coef;
  double* dred;
};

template <int R>
__device__ void cg_proj(float* v, const float* M, int n, const CgSmem& S) {
  float c[R];
#pragma unroll
  for (int t = 0; t < R; ++t) c[t] = 0.f;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    const float vq = v[q];
#pragma unroll
    for (int t = 0; t < R; ++t) c[t] = fmaf(M[q * R + t], vq, c[t]);
  }
  block_sum_R<R, kCgThreads>(c, S.red, S.coef);
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    float s = v[q];
#pragma unroll
    for (int t = 0; t < R; ++t) s = fmaf(-M[q * R + t], S.coef[t], s);
    v[q] = s;
  }
  __syncthreads();
}

// out(nI) = U v(nJ): one warp per row
__device__ void cg_mv(const float* __restrict__ U, int nI, int nJ, const float* v, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int row = warp; row < nI; row += kCgThreads / 32) {
    float s = 0.f;
    for (int b = lane; b < nJ; b += 32) s = fmaf(U[(size_t)row * nJ + b], v[b], s);
    s = warp_sum(s);
    if (lane == 0) out[row] = s;
  }
  __syncthreads();
}

// out(nJ) = U^T u(nI): one thread per column
__device__ void cg_mvt(const float* __restrict__ U, int nI, int nJ, const float* u, float* out) {
  for (int b = threadIdx.x; b < nJ; b += blockDim.x) {
    float s = 0.f;
    for (int row = 0; row < nI; ++row) s = fmaf(U[(size_t)row * nJ + b], u[row], s);
    out[b] = s;
  }
  __syncthreads();
}

__device__ double cg_dot(const float* x, const float* y, int n, const CgSmem& S) {
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += (double)x[q] * (double)y[q];
  return block_sum<kCgThreads>(s, S.dred);
}

size_t adj_cg_smem_bytes(int nI, int nJ, int Rpad) {
  const size_t f = (size_t)(nI + nJ) * Rpad + 6 * (size_t)nI + 6 * (size_t)nJ + (kCgThreads / 32) * Rpad + Rpad;
  return ((f * 4 + 15) & ~(size_t)15) + (kCgThreads / 32) * 8 + 16;
}

template <int R>
__global__ void __launch_bounds__(kCgThreads) adj_cg_kernel(AdjStep a) {
  extern __shared__ __align__(16) float sm[];
  const int nI = a.nI, nJ = a.nJ, i = blockIdx.x;
  CgSmem S;
  S.W = sm;
  S.V = S.W + (size_t)nI * R;
  S.phi = S.V + (size_t)nJ * R;
  S.rx = S.phi + nI;
  S.x = S.rx + nI;
  S.px = S.x + nI;
  S.apx = S.px + nI;
  S.tI = S.apx + nI;
  S.psi = S.tI + nI;
  S.ry = S.psi + nJ;
  S.y = S.ry + nJ;
  S.py = S.y + nJ;
  S.apy = S.py + nJ;
  S.tJ = S.apy + nJ;
  S.red = S.tJ + nJ;
  S.coef = S.red + (kCgThreads / 32) * R;
  {
    const size_t f = (size_t)(S.coef + R - sm);
    S.dred = reinterpret_cast<double*>(sm + ((f + 3) & ~(size_t)3));
  }
  for (int q = threadIdx.x; q < nI * R; q += blockDim.x) S.W[q] = a.Wr[q];
  for (int q = threadIdx.x; q < nJ * R; q += blockDim.x) S.V[q] = a.Vr[q];
  const float s = a.sig[i], s2 = s * s, inv = 1.f / s;
  // Phi_i = (R F^T) P(:,i) sigma_i,  Psi_i = (C^T E) P(:,i)
  for (int q = threadIdx.x; q < nI; q += blockDim.x) {
    float v = 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) v = fmaf(a.PhiY[q * R + t], a.Pm[t * R + i], v);
    S.phi[q] = v * s;
  }
  for (int q = threadIdx.x; q < nJ; q += blockDim.x) {
    float v = 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) v = fmaf(a.PsiY[q * R + t], a.Pm[t * R + i], v);
    S.psi[q] = v;
  }
  __syncthreads();
  // G11(:, i) = -(V_r^T Psi_i) / (sigma_t sigma_i)
  {
    float c[R];
#pragma unroll
    for (int t = 0; t < R; ++t) c[t] = 0.f;
    for (int q = threadIdx.x; q < nJ; q += blockDim.x) {
#pragma unroll
      for (int t = 0; t < R; ++t) c[t] = fmaf(S.V[q * R + t], S.psi[q], c[t]);
    }
    block_sum_R<R, kCgThreads>(c, S.red, S.coef);
    if (threadIdx.x < R) {
      const int t = threadIdx.x;
      const float st = a.sig[t];
      a.G11[t * R + i] = (t < a.r && st > 0.f) ? -S.coef[t] / (st * s) : 0.f;
    }
    __syncthreads();
  }
  // right-hand sides
  for (int q = threadIdx.x; q < nJ; q += blockDim.x) S.tJ[q] = S.psi[q];
  __syncthreads();
  cg_proj<R>(S.tJ, S.V, nJ, S);
  cg_mv(a.Ucore, nI, nJ, S.tJ, S.tI);
  for (int q = threadIdx.x; q < nI; q += blockDim.x) S.rx[q] = S.phi[q] + S.tI[q] * inv;
  __syncthreads();
  cg_proj<R>(S.rx, S.W, nI, S);
  for (int q = threadIdx.x; q < nI; q += blockDim.x) S.tI[q] = S.phi[q];
  __syncthreads();
  cg_proj<R>(S.tI, S.W, nI, S);
  cg_mvt(a.Ucore, nI, nJ, S.tI, S.tJ);
  for (int q = threadIdx.x; q < nJ; q += blockDim.x) S.ry[q] = S.psi[q] + S.tJ[q] * inv;
  __syncthreads();
  cg_proj<R>(S.ry, S.V, nJ, S);
  // CG on (s^2 - M_L) x = rx and (s^2 - M_R) y = ry
  for (int q = threadIdx.x; q < nI; q += blockDim.x) {
    S.x[q] = 0.f;
    S.px[q] = S.rx[q];
  }
  for (int q = threadIdx.x; q < nJ; q += blockDim.x) {
    S.y[q] = 0.f;
    S.py[q] = S.ry[q];
  }
  __syncthreads();
  double rsx = cg_dot(S.rx, S.rx, nI, S), rsy = cg_dot(S.ry, S.ry, nJ, S);
  const double rx0 = rsx, ry0 = rsy;
  const double tol2 = 1e-12;
  bool dx = rsx <= tol2 * rx0 || rx0 == 0.0, dy = rsy <= tol2 * ry0 || ry0 == 0.0;
  int it = 0;
  for (; it < a.cgMaxIter && !(dx && dy); ++it) {
    if (!dx) {  // apx = s^2 px - (1 - P_W) U (1 - P_V) U^T px
      cg_mvt(a.Ucore, nI, nJ, S.px, S.tJ);
      cg_proj<R>(S.tJ, S.V, nJ, S);
      cg_mv(a.Ucore, nI, nJ, S.tJ, S.tI);
      cg_proj<R>(S.tI, S.W, nI, S);
      for (int q = threadIdx.x; q < nI; q += blockDim.x) S.apx[q] = s2 * S.px[q] - S.tI[q];
      __syncthreads();
      const double pap = cg_dot(S.px, S.apx, nI, S);
      const float al = (float)(rsx / pap);
      for (int q = threadIdx.x; q < nI; q += blockDim.x) {
        S.x[q] = fmaf(al, S.px[q], S.x[q]);
        S.rx[q] = fmaf(-al, S.apx[q], S.rx[q]);
      }
      __syncthreads();
      const double rn = cg_dot(S.rx, S.rx, nI, S);
      const float be = (float)(rn / rsx);
      for (int q = threadIdx.x; q < nI; q += blockDim.x) S.px[q] = fmaf(be, S.px[q], S.rx[q]);
      __syncthreads();
      rsx = rn;
      dx = rsx <= tol2 * rx0;
    }
    if (!dy) {  // apy = s^2 py - (1 - P_V) U^T (1 - P_W) U py
      cg_mv(a.Ucore, nI, nJ, S.py, S.tI);
      cg_proj<R>(S.tI, S.W, nI, S);
      cg_mvt(a.Ucore, nI, nJ, S.tI, S.tJ);
      cg_proj<R>(S.tJ, S.V, nJ, S);
      for (int q = threadIdx.x; q < nJ; q += blockDim.x) S.apy[q] = s2 * S.py[q] - S.tJ[q];
      __syncthreads();
      const double pap = cg_dot(S.py, S.apy, nJ, S);
      const float al = (float)(rsy / pap);
      for (int q = threadIdx.x; q < nJ; q += blockDim.x) {
        S.y[q] = fmaf(al, S.py[q], S.y[q]);
        S.ry[q] = fmaf(-al, S.apy[q], S.ry[q]);
      }
      __syncthreads();
      const double rn = cg_dot(S.ry, S.ry, nJ, S);
      const float be = (float)(rn / rsy);
      for (int q = threadIdx.x; q < nJ; q += blockDim.x) S.py[q] = fmaf(be, S.py[q], S.ry[q]);
      __syncthreads();
      rsy = rn;
      dy = rsy <= tol2 * ry0;
    }
  }
  // A solve that stalled in FP32 is accepted once its residual fell by 1e-3;
  // otherwise the gap sigma_i > sigma_{r+1} is too small for the adjoint.
  const double accept2 = 1e-6;
  if (threadIdx.x == 0 && (rsx > accept2 * rx0 || rsy > accept2 * ry0)) atomicExch(a.status, (int)IRCUR_ESVD_NOCONV);
  for (int q = threadIdx.x; q < nI; q += blockDim.x) a.Xc[q * R + i] = S.x[q];
  for (int q = threadIdx.x; q < nJ; q += blockDim.x) a.Yc[q * R + i] = S.y[q];
}

// Ubar = W_r G11 V_r^T + Xs V_r^T + W_r Ys^T on row a; masked part GU to the
// scratch, the rest to dD(I_a, J); e1(a,:) += sum_b GU(a,b) B_k(:,J_b).
template <int R>
__global__ void __launch_bounds__(128) adj_core_finish_kernel(AdjStep a) {
  __shared__ float wh[R], wr[R], ar[R], red[4 * R], tot[R];
  const int row = blockIdx.x;
  if (threadIdx.x < R) {
    const int t = threadIdx.x;
    float v = a.Xc[row * R + t];
#pragma unroll
    for (int u = 0; u < R; ++u) v = fmaf(a.Wr[row * R + u], a.G11[u * R + t], v);
    wh[t] = v;
    wr[t] = a.Wr[row * R + t];
    ar[t] = a.Ak[(int64_t)a.I[row] * R + t];
  }
  __syncthreads();
  float acc[R];
#pragma unroll
  for (int t = 0; t < R; ++t) acc[t] = 0.f;
  for (int b = threadIdx.x; b < a.nJ; b += blockDim.x) {
    const int j = a.J[b];
    float ub = 0.f, bc[R], arr[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      ub = fmaf(wh[t], a.Vr[b * R + t], ub);
      ub = fmaf(wr[t], a.Yc[b * R + t], ub);
      bc[t] = a.Bk[(int64_t)t * a.n2 + j];
      arr[t] = ar[t];
    }
    const float l = lowrank_entry<R>(arr, bc);
    const float d = a.Prow[(int64_t)row * a.ldPr + j];
    const bool msk = fabsf(d - l) > a.zeta;
    const float gu = msk ? ub : 0.f;
    if (!msk) a.dDR[(int64_t)row * a.n2 + j] += ub;
    a.Ucore[(size_t)row * a.nJ + b] = gu;
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = fmaf(gu, bc[t], acc[t]);
  }
  block_sum_R<R, 128>(acc, red, tot);
  if (threadIdx.x < R) a.e1[row * R + threadIdx.x] += tot[threadIdx.x];
}

// f2(b,:) += sum_a GU(a,b) A_k(I_a,:)
template <int R>
__global__ void adj_core_cols_kernel(AdjStep a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.nJ) return;
  float acc[R];
#pragma unroll
  for (int t = 0; t < R; ++t) acc[t] = 0.f;
  for (int row = 0; row < a.nI; ++row) {
    const float g = a.Ucore[(size_t)row * a.nJ + b];
    const float* ar = a.Ak + (int64_t)a.I[row] * R;
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = fmaf(g, ar[t], acc[t]);
  }
#pragma unroll
  for (int t = 0; t < R; ++t) a.f2[b * R + t] += acc[t];
}

// E_k(I,:) += e1, F_k(:,J) += f2^T (index sets are distinct: no conflicts).
template <int R>
__global__ void adj_assemble_kernel(AdjStep a) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < a.nI * R) {
    const int row = q / R, t = q - row * R;
    a.Enew[(int64_t)a.I[row] * R + t] += a.e1[q];
  } else if (q < (a.nI + a.nJ) * R) {
    const int q2 = q - a.nI * R;
    const int b = q2 / R, t = q2 - b * R;
    a.Fnew[(int64_t)t * a.n2 + a.J[b]] += a.f2[q2];
  }
}

__global__ void adj_scatter_rows_kernel(const float* __restrict__ dDR, const int* __restrict__ I, int nI, int64_t n2,
                                        float* __restrict__ dD, int64_t lddD) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  if (j >= n2 || row >= nI) return;
  dD[(int64_t)I[row] * lddD + j] += dDR[(int64_t)row * n2 + j];
}

__global__ void adj_scatter_cols_kernel(const float* __restrict__ dDCt, const int* __restrict__ J, int nJ, int64_t n1,
                                        float* __restrict__ dD, int64_t lddD) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (i >= n1 || b >= nJ) return;
  dD[i * lddD + J[b]] += dDCt[(int64_t)b * n1 + i];
}

// ---------------------------------------------------------------------------
template <int R>
static cudaError_t launch_adj_dense_r(int64_t n1, int64_t n2, const float* A, const float* B, const float* D,
                                      int64_t ldD, const float* dL, int64_t lddL, const float* dS, int64_t lddS,
                                      float* dD, int64_t lddD, float zetaT, float* E, float* F, cudaStream_t s) {
  const unsigned rows_blocks = (unsigned)((n1 + kAdjThreads / 32 - 1) / (kAdjThreads / 32));
  adj_dense_rows_kernel<R><<<rows_blocks, kAdjThreads, 0, s>>>(n1, n2, A, B, D, ldD, dL, lddL, dS, lddS, dD, lddD,
                                                                zetaT, E);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned col_blocks = (unsigned)((n2 + kAdjCols - 1) / kAdjCols);
  adj_dense_cols_kernel<R><<<col_blocks, kAdjThreads, 0, s>>>(n1, n2, A, B, D, ldD, dL, lddL, dS, lddS, zetaT, F);
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_adj_step_r(const AdjStep& a, bool need_next, cudaStream_t s) {
  adj_small_kernel<R><<<1, kAdjThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    const int m = a.nI;
    const size_t bytes = (2 * (size_t)m * R + (size_t)kAdjSplit * kAdjCols * R) * 4;
    e = cudaFuncSetAttribute(adj_panel_kernel<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    adj_panel_kernel<R, false><<<a.nRowTiles, kAdjThreads, bytes, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  {
    const int m = a.nJ;
    const size_t bytes = (2 * (size_t)m * R + (size_t)kAdjSplit * kAdjCols * R) * 4;
    e = cudaFuncSetAttribute(adj_panel_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    adj_panel_kernel<R, true><<<a.nColTiles, kAdjThreads, bytes, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  adj_reduce_kernel<R><<<(a.nI * 2 * R + 255) / 256, 256, 0, s>>>(a.partR, a.nRowTiles, a.nI, a.PhiY, a.e1);
  adj_reduce_kernel<R><<<(a.nJ * 2 * R + 255) / 256, 256, 0, s>>>(a.partC, a.nColTiles, a.nJ, a.PsiY, a.f2);
  adj_core_build_kernel<R><<<a.nI, 128, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    const size_t bytes = adj_cg_smem_bytes(a.nI, a.nJ, R);
    e = cudaFuncSetAttribute(adj_cg_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    adj_cg_kernel<R><<<a.r, kCgThreads, bytes, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  adj_core_finish_kernel<R><<<a.nI, 128, 0, s>>>(a);
  adj_core_cols_kernel<R><<<(a.nJ + 127) / 128, 128, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (need_next) {
    adj_assemble_kernel<R><<<((a.nI + a.nJ) * R + 255) / 256, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

#define IRCUR_ADJ_DISPATCH(FN, ...)             \
  switch (Rpad) {                               \
    case 1: return FN<1>(__VA_ARGS__);          \
    case 2: return FN<2>(__VA_ARGS__);          \
    case 3: return FN<3>(__VA_ARGS__);          \
    case 4: return FN<4>(__VA_ARGS__);          \
    case 5: return FN<5>(__VA_ARGS__);          \
    case 6: return FN<6>(__VA_ARGS__);          \
    case 7: return FN<7>(__VA_ARGS__);          \
    case 8: return FN<8>(__VA_ARGS__);          \
    case 9: return FN<9>(__VA_ARGS__);          \
    case 10: return FN<10>(__VA_ARGS__);        \
    case 12: return FN<12>(__VA_ARGS__);        \
    case 16: return FN<16>(__VA_ARGS__);        \
    case 20: return FN<20>(__VA_ARGS__);        \
    default: return cudaErrorInvalidValue;      \
  }

cudaError_t launch_adj_dense(int64_t n1, int64_t n2, const float* A, const float* B, const float* D, int64_t ldD,
                             const float* dL, int64_t lddL, const float* dS, int64_t lddS, float* dD,
                             int64_t lddD, float zetaT, float* E, float* F, int Rpad, cudaStream_t s) {
  IRCUR_ADJ_DISPATCH(launch_adj_dense_r, n1, n2, A, B, D, ldD, dL, lddL, dS, lddS, dD, lddD, zetaT, E, F, s)
}

cudaError_t launch_adj_step(const AdjStep& a, int Rpad, bool need_next, cudaStream_t s) {
  IRCUR_ADJ_DISPATCH(launch_adj_step_r, a, need_next, s)
}

cudaError_t launch_adj_scatter(const AdjStep& a, float* dD, int64_t lddD, cudaStream_t s) {
  adj_scatter_rows_kernel<<<dim3((unsigned)((a.n2 + 255) / 256), a.nI), 256, 0, s>>>(a.dDR, a.I, a.nI, a.n2, dD,
                                                                                     lddD);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  adj_scatter_cols_kernel<<<dim3((unsigned)((a.n1 + 255) / 256), a.nJ), 256, 0, s>>>(a.dDCt, a.J, a.nJ, a.n1, dD,
                                                                                     lddD);
  return cudaGetLastError();
}

}  // namespace ircur
