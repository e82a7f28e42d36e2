// CUR to SVD (Alg. 2) for the iterate the solver holds, L = A B with
// A = C X T^{-1} (n1 x r) and B = Y^T R (r x n2):
//   A = Q_A R_A  (R_A^T R_A = A^T A),   B^T = Q_B R_B  (R_B^T R_B = B B^T),
//   L = Q_A (R_A R_B^T) Q_B^T,   R_A R_B^T = P Sigma Q^T  (an r x r SVD),
//   W = Q_A P = A (R_A^{-1} P),  V = Q_B Q = B^T (R_B^{-1} Q).
// Alg. 2 takes the QRs of C and R^T and the SVD of R_C U^+ R_R^T; on the
// factored iterate the same singular triplets follow from the two skinny
// factors, with Q_A and Q_B never formed: one Gram pass over A and B
// (FP64 accumulation), the r x r algebra in FP64 in one block, and one pass
// writing W and V.
#include <float.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

constexpr int kGramChunk = 256;  // rows of A (columns of B) per block of the Gram pass

// Block b < nbA: A^T A over rows [b c, (b+1) c) of A; block nbA + b: B B^T over
// columns [b c, (b+1) c) of B.  Thread (s, t) owns entry (s, t).
template <int R>
__global__ void c2s_gram_kernel(const float* __restrict__ A, int64_t n1, const float* __restrict__ B, int64_t n2,
                                int nbA, double* __restrict__ part) {
  const int q = threadIdx.x;
  if (q >= R * R) return;
  const int s = q / R, t = q - s * R;
  double acc = 0.0;
  if ((int)blockIdx.x < nbA) {
    const int64_t i0 = (int64_t)blockIdx.x * kGramChunk;
    const int64_t i1 = i0 + kGramChunk < n1 ? i0 + kGramChunk : n1;
    for (int64_t i = i0; i < i1; ++i) acc = fma((double)A[i * R + s], (double)A[i * R + t], acc);
  } else {
    const int64_t j0 = (int64_t)(blockIdx.x - nbA) * kGramChunk;
    const int64_t j1 = j0 + kGramChunk < n2 ? j0 + kGramChunk : n2;
    for (int64_t j = j0; j < j1; ++j) acc = fma((double)B[(int64_t)s * n2 + j], (double)B[(int64_t)t * n2 + j], acc);
  }
  part[(size_t)blockIdx.x * R * R + q] = acc;
}

// Upper Cholesky factor of the r x r SPD matrix G (FP64, one warp, lane =
// row); pivots <= 1e-13 of the largest diagonal entry give zero rows.
template <int R>
__device__ void c2s_chol(const double* G, int r, double* U) {
  const int lane = threadIdx.x & 31;
  double g[R];
#pragma unroll
  for (int u = 0; u < R; ++u) g[u] = (lane < r && u < r) ? G[lane * R + u] : 0.0;
  double dmax = 0.0;
#pragma unroll
  for (int u = 0; u < R; ++u)
    if (u == lane) dmax = g[u];
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  for (int t = 0; t < r; ++t) {
    double gt = 0.0;
#pragma unroll
    for (int u = 0; u < R; ++u)
      if (u == t) gt = g[u];
    const double dgt = __shfl_sync(0xffffffffu, gt, t);
    const double rinv = dgt > 1e-13 * dmax ? 1.0 / sqrt(dgt) : 0.0;
    const double ul = gt * rinv;  // U(t, lane)
    double urow[R];
#pragma unroll
    for (int u = 0; u < R; ++u) urow[u] = __shfl_sync(0xffffffffu, ul, u);
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < R; ++u) U[t * R + u] = (u >= t && u < r) ? urow[u] : 0.0;
    }
    if (lane > t) {
#pragma unroll
      for (int u = 0; u < R; ++u) g[u] = fma(-ul, urow[u], g[u]);
    }
  }
  if (lane == 0)
    for (int t = r; t < R; ++t)
      for (int u = 0; u < R; ++u) U[t * R + u] = 0.0;
  __syncwarp();
}

// X = U^{-1} Y for upper-triangular U (zero pivots give zero rows), column c per lane.
template <int R>
__device__ void c2s_backsolve(const double* U, const double* Y, int r, double* X) {
  const int c = threadIdx.x & 31;
  if (c < r) {
    double x[R];
#pragma unroll
    for (int s2 = R - 1; s2 >= 0; --s2) {
      double v = 0.0;
      if (s2 < r && U[s2 * R + s2] != 0.0) {
        v = Y[s2 * R + c];
#pragma unroll
        for (int u = s2 + 1; u < R; ++u)
          if (u < r) v = fma(-U[s2 * R + u], x[u], v);
        v = v / U[s2 * R + s2];
      }
      x[s2] = v;
    }
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) X[s2 * R + c] = x[s2];
  }
  __syncwarp();
}

// One block: fixed-order sums of the Gram partials, the two Cholesky factors,
// M = R_A R_B^T, its SVD by one-sided Jacobi (lane p owns column p of M and of
// the rotation Q), and the r x r maps T_A = R_A^{-1} P, T_B = R_B^{-1} Q with
// the singular values sorted in descending order.
// (launched with R * R threads, at least a warp: the bound keeps R = 20's 400
// threads within the register file)
template <int R>
__global__ void __launch_bounds__(R * R < 32 ? 32 : R * R)
    c2s_small_kernel(const double* __restrict__ part, int nbA, int nbB, int r, float* __restrict__ sigma,
                                 float* __restrict__ TA, float* __restrict__ TB) {
  __shared__ double GA[R * R], GB[R * R], RA[R * R], RB[R * R], P[R * R], Q[R * R], XA[R * R], XB[R * R];
  __shared__ double sg[R];
  const int q = threadIdx.x;
  if (q < R * R) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nbA; ++k) a += part[(size_t)k * R * R + q];
    for (int k = 0; k < nbB; ++k) b += part[(size_t)(nbA + k) * R * R + q];
    GA[q] = a;
    GB[q] = b;
  }
  __syncthreads();
  if (q < 32) {
    c2s_chol<R>(GA, r, RA);
    c2s_chol<R>(GB, r, RB);
    // M = R_A R_B^T; lane p holds column p of M and of Q (identity to start)
    const int p = q;
    double mc[R], qc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      double v = 0.0;
      if (p < r && i < r)
        for (int u = 0; u < r; ++u) v = fma(RA[i * R + u], RB[p * R + u], v);
      mc[i] = v;
      qc[i] = (p < r && i == p) ? 1.0 : 0.0;
    }
    const int nplay = (r + 1) & ~1;
    for (int sweep = 0; sweep < 60; ++sweep) {
      int rotated = 0;
      for (int rnd = 0; rnd < nplay - 1; ++rnd) {
        int o = p;  // circle-method partner
        if (p < nplay) {
          const int m = nplay - 1;
          if (p == m)
            o = rnd;
          else if (p == rnd)
            o = m;
          else
            o = (2 * rnd - p + 2 * m) % m;
        }
        double mo[R], qo[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
          mo[i] = __shfl_sync(0xffffffffu, mc[i], o);
          qo[i] = __shfl_sync(0xffffffffu, qc[i], o);
        }
        if (p < r && o < r && o != p) {
          const bool lo = p < o;
          double app = 0.0, aoo = 0.0, apo = 0.0;
#pragma unroll
          for (int i = 0; i < R; ++i) {
            const double x = lo ? mc[i] : mo[i], y = lo ? mo[i] : mc[i];
            app = fma(x, x, app);
            aoo = fma(y, y, aoo);
            apo = fma(x, y, apo);
          }
          if (fabs(apo) > 1e-15 * sqrt(app * aoo)) {
            rotated = 1;
            const double zz = (aoo - app) / (2.0 * apo);
            const double tt = copysign(1.0, zz) / (fabs(zz) + sqrt(1.0 + zz * zz));
            const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const double x = lo ? mc[i] : mo[i], y = lo ? mo[i] : mc[i];
              mc[i] = lo ? (cs * x - sn * y) : (sn * x + cs * y);
              const double u = lo ? qc[i] : qo[i], v = lo ? qo[i] : qc[i];
              qc[i] = lo ? (cs * u - sn * v) : (sn * u + cs * v);
            }
          }
        }
      }
      if (!__any_sync(0xffffffffu, rotated)) break;
    }
    double n2s = 0.0;
#pragma unroll
    for (int i = 0; i < R; ++i) n2s = fma(mc[i], mc[i], n2s);
    const double sgv = p < r ? sqrt(n2s) : -1.0;
    // descending order (ties: smaller index first)
    int pos = 0;
    for (int o = 0; o < r; ++o) {
      const double so = __shfl_sync(0xffffffffu, sgv, o);
      pos += (so > sgv) || (so == sgv && o < p);
    }
    if (p < r) {
      sg[pos] = sgv;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        P[i * R + pos] = sgv > 0.0 ? mc[i] / sgv : 0.0;
        Q[i * R + pos] = qc[i];
      }
    }
    __syncwarp();
    if (p < R && p >= r) {
#pragma unroll
      for (int i = 0; i < R; ++i) {
        P[i * R + p] = 0.0;
        Q[i * R + p] = 0.0;
      }
    }
    __syncwarp();
    c2s_backsolve<R>(RA, P, r, XA);
    c2s_backsolve<R>(RB, Q, r, XB);
  }
  __syncthreads();
  if (q < R * R) {
    TA[q] = (float)XA[q];
    TB[q] = (float)XB[q];
  }
  if (q < r) sigma[q] = (float)sg[q];
}

// W = A T_A (n1 x r, row-major, ld r) and V = B^T T_B (n2 x r): one row per thread.
template <int R>
__global__ void c2s_apply_kernel(const float* __restrict__ A, int64_t n1, const float* __restrict__ B, int64_t n2,
                                 int r, const float* __restrict__ TA, const float* __restrict__ TB,
                                 float* __restrict__ W, float* __restrict__ V) {
  __shared__ float ta[R * R], tb[R * R];
  for (int q = threadIdx.x; q < R * R; q += blockDim.x) {  // R * R may exceed the block
    ta[q] = TA[q];
    tb[q] = TB[q];
  }
  __syncthreads();
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n1) {
    float a[R];
#pragma unroll
    for (int s = 0; s < R; ++s) a[s] = A[idx * R + s];
    for (int t = 0; t < r; ++t) {
      float v = 0.f;
#pragma unroll
      for (int s = 0; s < R; ++s) v = fmaf(a[s], ta[s * R + t], v);
      W[idx * r + t] = v;
    }
  } else if (idx < n1 + n2) {
    const int64_t j = idx - n1;
    float b[R];
#pragma unroll
    for (int s = 0; s < R; ++s) b[s] = B[(int64_t)s * n2 + j];
    for (int t = 0; t < r; ++t) {
      float v = 0.f;
#pragma unroll
      for (int s = 0; s < R; ++s) v = fmaf(b[s], tb[s * R + t], v);
      V[j * r + t] = v;
    }
  }
}

size_t cur_to_svd_scratch_bytes(int64_t n1, int64_t n2, int Rpad) {
  const int64_t nbA = (n1 + kGramChunk - 1) / kGramChunk, nbB = (n2 + kGramChunk - 1) / kGramChunk;
  return (size_t)(nbA + nbB) * Rpad * Rpad * 8 + 2 * (size_t)Rpad * Rpad * 4 + 256;
}

template <int R>
static cudaError_t launch_c2s_r(const float* A, const float* B, int64_t n1, int64_t n2, int r, void* scratch,
                                float* W, float* sigma, float* V, cudaStream_t s) {
  const int nbA = (int)((n1 + kGramChunk - 1) / kGramChunk), nbB = (int)((n2 + kGramChunk - 1) / kGramChunk);
  double* part = static_cast<double*>(scratch);
  float* TA = reinterpret_cast<float*>(part + (size_t)(nbA + nbB) * R * R);
  float* TB = TA + R * R;
  c2s_gram_kernel<R><<<nbA + nbB, R * R < 32 ? 32 : R * R, 0, s>>>(A, n1, B, n2, nbA, part);
  c2s_small_kernel<R><<<1, R * R < 32 ? 32 : R * R, 0, s>>>(part, nbA, nbB, r, sigma, TA, TB);
  const int64_t rows = n1 + n2;
  c2s_apply_kernel<R><<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(A, n1, B, n2, r, TA, TB, W, V);
  return cudaGetLastError();
}

cudaError_t launch_cur_to_svd(const float* A, const float* B, int64_t n1, int64_t n2, int r, int Rpad, void* scratch,
                              float* W, float* sigma, float* V, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_c2s_r<1>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 2: return launch_c2s_r<2>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 3: return launch_c2s_r<3>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 4: return launch_c2s_r<4>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 5: return launch_c2s_r<5>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 6: return launch_c2s_r<6>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 7: return launch_c2s_r<7>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 8: return launch_c2s_r<8>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 9: return launch_c2s_r<9>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 10: return launch_c2s_r<10>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 12: return launch_c2s_r<12>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 16: return launch_c2s_r<16>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    case 20: return launch_c2s_r<20>(A, B, n1, n2, r, scratch, W, sigma, V, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ircur
