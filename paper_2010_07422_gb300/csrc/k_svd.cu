// Rank-r truncation H_r of the |I| x |J| core and its pseudo-inverse
// (Alg. 1 Phase II; Sec. 3.1: U_{k+1} = H_r([D - S_{k+1}]_{I,J}),
// U^+ = V_r Sigma_r^{-1} W_r^T).
//
// One CTA of 512 threads.  The dominant rank-r singular subspaces are found
// by two-sided subspace (orthogonal) iteration with Cholesky-QR, warm-started
// from the previous iterate's right factor B_k(:,J)^T, whose row space is the
// right singular subspace of L_k(I,J); the core of iteration k+1 differs from
// L_k(I,J) only by the change of the thresholded entries.  Each step is
//     P = core X,  Y Rc = P (CholQR),  Q = core^T Y,
// and stops once the residual E = Q - X Rc^T (the part of core^T Y outside
// span X) is below 1e-6 ||Rc||_F, or stagnates below 1e-4 ||Rc||_F.  The r x r
// Rayleigh-Ritz matrix T = Y^T core X is then diagonalised by a one-sided
// Jacobi SVD in one warp, giving W_r = Y U_T, V_r = X V_T, sigma_r.
// Singular values <= max(|I|,|J|) * FLT_EPSILON * sigma_1 are dropped
// (numerical rank; IRCUR_FLAG_WRANK).
//
// Precision: the core and the m-long products are FP32; Gram matrices are
// accumulated per lane in FP32 and across lanes in FP64, and the Cholesky
// factorisation and triangular inverse run in FP64.
#include <float.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

constexpr int kSvdThreads = 512;

__host__ __device__ constexpr int round_up4(int x) { return (x + 3) & ~3; }

struct SvdLayout {
  int ldu;       // leading dimension of the core copy in shared memory (odd)
  int rx;        // row stride of the m x R blocks (R rounded up to 4)
  int mmax;      // max(nI, nJ)
  size_t off_us, off_x, off_y, off_p, off_q, off_part, off_small, total;
};

__host__ __device__ inline SvdLayout svd_layout(int nI, int nJ, int R, bool core_in_smem) {
  SvdLayout L;
  L.ldu = nJ | 1;
  L.rx = round_up4(R);
  L.mmax = nI > nJ ? nI : nJ;
  size_t off = 0;
  L.off_us = off;
  if (core_in_smem) off += (size_t)nI * L.ldu * 4;
  off = (off + 15) & ~(size_t)15;
  L.off_x = off;
  off += (size_t)L.mmax * L.rx * 4;
  L.off_y = off;
  off += (size_t)L.mmax * L.rx * 4;
  L.off_p = off;
  off += (size_t)L.mmax * L.rx * 4;
  L.off_q = off;
  off += (size_t)L.mmax * L.rx * 4;
  L.off_part = off;
  off += (size_t)kSvdThreads * L.rx * 4;
  L.off_small = off;
  // G, Rc (double R*R each), Rinv, T, Ut, Vt (float R*R each), sig, scalars
  off += 2 * (size_t)R * R * 8 + 4 * (size_t)R * R * 4 + 64 * 4 + 256;
  L.total = (off + 15) & ~(size_t)15;
  return L;
}

size_t svd_smem_bytes(int nI, int nJ, int Rpad, bool* core_in_smem) {
  SvdLayout L = svd_layout(nI, nJ, Rpad, true);
  if (L.total <= 220 * 1024) {
    *core_in_smem = true;
    return L.total;
  }
  *core_in_smem = false;
  return svd_layout(nI, nJ, Rpad, false).total;
}

struct SvdSmall {
  double* G;     // R x R Gram
  double* Rc;    // R x R upper Cholesky factor
  float* Rinv;   // R x R inverse of Rc (zero rows/cols for dropped pivots)
  float* T;      // R x R Rayleigh-Ritz matrix
  float* Ut;     // R x R
  float* Vt;     // R x R
  float* sig;    // R
  float* red;    // 32 reduction slots
  int* ibuf;     // 8 ints
};

// out(o, t) = sum_q U(o, q) in(q, t), U = core (nI x nJ) or its transpose.
// Threads are laid out as (chunk, row): the inner index range is split in
// nch chunks whose partial sums are added in a fixed order (deterministic).
template <int R>
__device__ void core_product(const float* __restrict__ U, int ldu, bool transposed, int nout, int nin,
                             const float* __restrict__ in, float* __restrict__ out, float* part, int rx) {
  const int rows32 = (nout + 31) & ~31;
  const int nch = blockDim.x / rows32 > 0 ? (int)(blockDim.x / rows32) : 1;
  const int c = threadIdx.x / rows32, o = threadIdx.x % rows32;
  if (c < nch && o < nout) {
    float acc[R];
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = 0.f;
    const int q0 = (int)((long long)c * nin / nch), q1 = (int)((long long)(c + 1) * nin / nch);
    for (int q = q0; q < q1; ++q) {
      const float u = transposed ? U[(size_t)q * ldu + o] : U[(size_t)o * ldu + q];
      const float* m = in + (size_t)q * rx;
#pragma unroll
      for (int t = 0; t < R; ++t) acc[t] = fmaf(u, m[t], acc[t]);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) part[((size_t)c * rows32 + o) * rx + t] = acc[t];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nout * R; idx += blockDim.x) {
    const int oo = idx / R, t = idx % R;
    float s = 0.f;
    for (int cc = 0; cc < nch; ++cc) s += part[((size_t)cc * rows32 + oo) * rx + t];
    out[(size_t)oo * rx + t] = s;
  }
  __syncthreads();
}

// In-place Cholesky QR of the nrows x r block M (stride rx): M <- M Rc^{-1},
// Rc (FP64, upper) with M_in = M_out Rc.  Pivots below 1e-10 of the largest
// diagonal entry are treated as dependent columns: they become zero columns
// and count as breakdowns (returned).
template <int R>
__device__ int cholqr(float* M, int nrows, int r, int rx, const SvdSmall& sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int npairs = r * (r + 1) / 2;
  for (int p = warp; p < npairs; p += nwarps) {
    int s = 0, rem = p;
    while (rem >= r - s) {
      rem -= r - s;
      ++s;
    }
    const int t = s + rem;
    float acc = 0.f;
    for (int i = lane; i < nrows; i += 32) acc = fmaf(M[(size_t)i * rx + s], M[(size_t)i * rx + t], acc);
    const double tot = warp_sum((double)acc);
    if (lane == 0) {
      sm.G[s * R + t] = tot;
      sm.G[t * R + s] = tot;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double maxd = 0.0;
    for (int t = 0; t < r; ++t) maxd = fmax(maxd, sm.G[t * R + t]);
    int brk = 0;
    for (int s = 0; s < R; ++s)
      for (int t = 0; t < R; ++t) sm.Rc[s * R + t] = 0.0;
    for (int t = 0; t < r; ++t) {
      double dg = sm.G[t * R + t];
      for (int s = 0; s < t; ++s) dg -= sm.Rc[s * R + t] * sm.Rc[s * R + t];
      if (!(dg > 1e-10 * maxd) || !(maxd > 0.0)) {
        ++brk;
        continue;  // dependent column: zero row of Rc
      }
      const double d = sqrt(dg);
      sm.Rc[t * R + t] = d;
      for (int u = t + 1; u < r; ++u) {
        double v = sm.G[t * R + u];
        for (int s = 0; s < t; ++s) v -= sm.Rc[s * R + t] * sm.Rc[s * R + u];
        sm.Rc[t * R + u] = v / d;
      }
    }
    // inverse of the upper-triangular Rc (skipping dropped pivots)
    double inv[R * R];
    for (int s = 0; s < R * R; ++s) inv[s] = 0.0;
    for (int t = 0; t < r; ++t) {
      if (sm.Rc[t * R + t] == 0.0) continue;
      inv[t * R + t] = 1.0 / sm.Rc[t * R + t];
      for (int s = t - 1; s >= 0; --s) {
        if (sm.Rc[s * R + s] == 0.0) continue;
        double v = 0.0;
        for (int u = s + 1; u <= t; ++u) v += sm.Rc[s * R + u] * inv[u * R + t];
        inv[s * R + t] = -v / sm.Rc[s * R + s];
      }
    }
    for (int s = 0; s < R * R; ++s) sm.Rinv[s] = (float)inv[s];
    sm.ibuf[0] = brk;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    float m[R], o[R];
#pragma unroll
    for (int s = 0; s < R; ++s) m[s] = M[(size_t)i * rx + s];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float v = 0.f;
#pragma unroll
      for (int s = 0; s <= t; ++s) v = fmaf(m[s], sm.Rinv[s * R + t], v);
      o[t] = v;
    }
#pragma unroll
    for (int t = 0; t < R; ++t) M[(size_t)i * rx + t] = o[t];
  }
  const int brk = sm.ibuf[0];
  __syncthreads();
  return brk;
}

__device__ float block_sum(float v, float* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    red[31] = s;
  }
  __syncthreads();
  s = red[31];
  __syncthreads();
  return s;
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

template <int R>
__global__ void __launch_bounds__(kSvdThreads) svd_kernel(IterDesc d, int core_in_smem) {
  State* st = d.st;
  if (st->done || st->status) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int k = st->k;
  const int cur = k & 1;
  const int nI = d.nI, nJ = d.nJ, r = d.r;
  const int* J = d.J_all + (d.resample ? (int64_t)k * nJ : 0);
  const SvdLayout L = svd_layout(nI, nJ, R, core_in_smem != 0);
  const int rx = L.rx;
  float* Us = core_in_smem ? reinterpret_cast<float*>(smem + L.off_us) : d.core;
  const int ldu = core_in_smem ? L.ldu : nJ;
  float* X = reinterpret_cast<float*>(smem + L.off_x);
  float* Y = reinterpret_cast<float*>(smem + L.off_y);
  float* P = reinterpret_cast<float*>(smem + L.off_p);
  float* Q = reinterpret_cast<float*>(smem + L.off_q);
  float* part = reinterpret_cast<float*>(smem + L.off_part);
  SvdSmall sm;
  {
    unsigned char* p = smem + L.off_small;
    sm.G = reinterpret_cast<double*>(p);
    p += (size_t)R * R * 8;
    sm.Rc = reinterpret_cast<double*>(p);
    p += (size_t)R * R * 8;
    sm.Rinv = reinterpret_cast<float*>(p);
    p += (size_t)R * R * 4;
    sm.T = reinterpret_cast<float*>(p);
    p += (size_t)R * R * 4;
    sm.Ut = reinterpret_cast<float*>(p);
    p += (size_t)R * R * 4;
    sm.Vt = reinterpret_cast<float*>(p);
    p += (size_t)R * R * 4;
    sm.sig = reinterpret_cast<float*>(p);
    p += 32 * 4;
    sm.red = reinterpret_cast<float*>(p);
    p += 32 * 4;
    sm.ibuf = reinterpret_cast<int*>(p);
  }

  // ---- core into shared memory (odd leading dimension: conflict-free columns)
  if (core_in_smem) {
    for (int q = threadIdx.x; q < nI * nJ; q += blockDim.x) {
      const int i = q / nJ, j = q - i * nJ;
      Us[(size_t)i * ldu + j] = d.core[q];
    }
  }
  // ---- warm start X = B_k(:,J)^T (zero columns t >= r)
  const float* Bk = d.B[cur];
  for (int q = threadIdx.x; q < nJ * rx; q += blockDim.x) {
    const int b = q / rx, t = q - b * rx;
    X[q] = (t < r) ? Bk[(int64_t)t * d.n2 + J[b]] : 0.f;
  }
  __syncthreads();
  int brk = cholqr<R>(X, nJ, r, rx, sm);
  if (brk > 0) {  // first iteration (B_0 = 0) or a deficient factor: random start
    for (int q = threadIdx.x; q < nJ * rx; q += blockDim.x) {
      const int t = q % rx;
      X[q] = (t < r) ? hash_uniform(d.seed ^ 0x5bd1e995ull, ((uint64_t)k << 32) ^ (uint64_t)q) : 0.f;
    }
    __syncthreads();
    cholqr<R>(X, nJ, r, rx, sm);
  }

  // ---- subspace iteration
  int steps = 0;
  bool converged = false;
  float prev_res = 0.f;
  while (steps < d.svdMaxSteps) {
    ++steps;
    core_product<R>(Us, ldu, false, nI, nJ, X, Y, part, rx);  // Y = core X
    cholqr<R>(Y, nI, r, rx, sm);                               // Y Rc = core X
    core_product<R>(Us, ldu, true, nJ, nI, Y, Q, part, rx);    // Q = core^T Y
    // E = Q - X Rc^T ; ||E||_F^2 and ||Rc||_F^2
    float e2 = 0.f;
    for (int q = threadIdx.x; q < nJ * r; q += blockDim.x) {
      const int b = q / r, t = q - b * r;
      float v = Q[(size_t)b * rx + t];
      for (int s = t; s < r; ++s) v -= X[(size_t)b * rx + s] * (float)sm.Rc[t * R + s];
      e2 = fmaf(v, v, e2);
    }
    float rc2 = 0.f;
    if (threadIdx.x < R * R) {
      const float v = (float)sm.Rc[threadIdx.x];
      rc2 = v * v;
    }
    const float E2 = block_sum(e2, sm.red);
    const float RC2 = block_sum(rc2, sm.red);
    const float res = sqrtf(E2), nrm = sqrtf(RC2);
    if (res <= 1e-6f * nrm || (steps > 1 && res > 0.5f * prev_res && res <= 1e-4f * nrm) || !(nrm > 0.f)) {
      converged = true;
      break;
    }
    prev_res = res;
    for (int q = threadIdx.x; q < nJ * rx; q += blockDim.x) X[q] = Q[q];
    __syncthreads();
    cholqr<R>(X, nJ, r, rx, sm);
  }

  // ---- final bases: X re-orthonormalised, Y = orth(core X) twice, T = Y^T core X
  cholqr<R>(X, nJ, r, rx, sm);
  core_product<R>(Us, ldu, false, nI, nJ, X, P, part, rx);  // P = core X
  for (int q = threadIdx.x; q < nI * rx; q += blockDim.x) Y[q] = P[q];
  __syncthreads();
  cholqr<R>(Y, nI, r, rx, sm);
  cholqr<R>(Y, nI, r, rx, sm);
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int p = warp; p < r * r; p += nwarps) {
      const int s = p / r, t = p % r;
      float acc = 0.f;
      for (int i = lane; i < nI; i += 32) acc = fmaf(Y[(size_t)i * rx + s], P[(size_t)i * rx + t], acc);
      acc = warp_sum(acc);
      if (lane == 0) sm.T[s * R + t] = acc;
    }
  }
  __syncthreads();

  // ---- one-sided Jacobi SVD of T (r x r) in warp 0: lane p owns column p
  if (threadIdx.x < 32) {
    const int p = threadIdx.x;
    float tc[R], vc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      tc[i] = (p < r && i < r) ? sm.T[i * R + p] : 0.f;
      vc[i] = (i == p) ? 1.f : 0.f;
    }
    const int nplay = (r + 1) & ~1;
    for (int sweep = 0; sweep < 40; ++sweep) {
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
          if (fabsf(apq) > 1e-7f * sqrtf(app * aqq) && apq != 0.f) {
            rotated = 1;
            const float zeta = (aqq - app) / (2.f * apq);
            const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
            const float c = 1.f / sqrtf(1.f + tt * tt), s = c * tt;
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const float a = lo ? tc[i] : tq[i], b = lo ? tq[i] : tc[i];
              const float va = lo ? vc[i] : vq[i], vb = lo ? vq[i] : vc[i];
              tc[i] = lo ? (c * a - s * b) : (s * a + c * b);
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
    const float sg = (p < r) ? sqrtf(s2) : -1.f;
    int pos = 0;
    for (int q = 0; q < r; ++q) {
      const float sq = __shfl_sync(0xffffffffu, sg, q);
      pos += (sq > sg) || (sq == sg && q < p);
    }
    if (p < r) {
      const float inv = sg > 0.f ? 1.f / sg : 0.f;
#pragma unroll
      for (int i = 0; i < R; ++i) {
        sm.Ut[i * R + pos] = tc[i] * inv;
        sm.Vt[i * R + pos] = vc[i];
      }
      sm.sig[pos] = sg;
    }
  }
  __syncthreads();
  // numerical rank
  if (threadIdx.x == 0) {
    const float s0 = sm.sig[0];
    const float tol = (float)(nI > nJ ? nI : nJ) * FLT_EPSILON * s0;
    int rank = 0;
    for (int t = 0; t < r; ++t) rank += sm.sig[t] > tol && sm.sig[t] > 0.f;
    sm.ibuf[1] = rank;
    for (int t = r; t < R; ++t) sm.sig[t] = 0.f;
  }
  __syncthreads();
  const int rank = sm.ibuf[1];
  // W = Y Ut (nI x R), V = X Vt, Vs = V / sigma; zero columns beyond the rank
  for (int q = threadIdx.x; q < nI * R; q += blockDim.x) {
    const int i = q / R, t = q - i * R;
    float v = 0.f;
    if (t < rank)
      for (int s = 0; s < r; ++s) v = fmaf(Y[(size_t)i * rx + s], sm.Ut[s * R + t], v);
    d.W[q] = v;
  }
  for (int q = threadIdx.x; q < nJ * R; q += blockDim.x) {
    const int b = q / R, t = q - b * R;
    float v = 0.f;
    if (t < rank)
      for (int s = 0; s < r; ++s) v = fmaf(X[(size_t)b * rx + s], sm.Vt[s * R + t], v);
    d.V[q] = v;
    d.Vs[q] = (t < rank) ? v / sm.sig[t] : 0.f;
  }
  if (threadIdx.x < R) d.sigma[threadIdx.x] = (threadIdx.x < rank) ? sm.sig[threadIdx.x] : 0.f;
  if (threadIdx.x == 0) {
    unsigned f = 0u;
    if (rank < r) f |= IRCUR_FLAG_WRANK;
    if (!converged) f |= IRCUR_FLAG_SVD_NOCONV;
    if (f) atomicOr(&st->flags, f);
    st->svd_steps += steps;
    st->svd_last_steps = steps;
  }
}

template <int R>
static cudaError_t launch_svd_r(const IterDesc& d, cudaStream_t s) {
  bool in_smem = false;
  const size_t bytes = svd_smem_bytes(d.nI, d.nJ, R, &in_smem);
  cudaError_t e = cudaFuncSetAttribute(svd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  svd_kernel<R><<<1, kSvdThreads, bytes, s>>>(d, in_smem ? 1 : 0);
  return cudaGetLastError();
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
