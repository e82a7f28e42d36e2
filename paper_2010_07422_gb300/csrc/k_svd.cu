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
// Then Y and X get a second CholQR pass, the r x r Rayleigh-Ritz matrix
// T = Y^T core X follows from the triangular factors without another
// product, and a one-sided Jacobi SVD of T in one warp gives
// W_r = Y U_T, V_r = X V_T and sigma_r.  Singular values
// <= max(|I|,|J|) * FLT_EPSILON * sigma_1 are dropped (numerical rank,
// IRCUR_FLAG_WRANK).
//
// Precision: FP32 throughout.  GB300's FP64 pipe runs at a small fraction of
// its FP32 rate, and the serial FP64 Cholesky/sqrt/divide chains of a first
// version cost more than the whole rest of the iteration; CholQR2 (the
// second pass) restores orthogonality to FP32 rounding.
#include <float.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

constexpr int kSvdThreads = 512;

__host__ __device__ constexpr int round_up4(int x) { return (x + 3) & ~3; }

struct SvdLayout {
  int ldu;   // leading dimension of the core copy in shared memory (odd)
  int rx;    // row stride of the m x R blocks (R rounded up to 4)
  int mmax;  // max(nI, nJ)
  size_t off_us, off_x, off_y, off_q, off_part, off_small, total;
};

constexpr int kSmallMats = 9;  // G, Rp, U, U2y, U2x, T, Ut, Vt, scratch (R x R each)

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
  L.off_q = off;
  off += (size_t)L.mmax * L.rx * 4;
  L.off_part = off;
  off += (size_t)kSvdThreads * L.rx * 4;
  L.off_small = off;
  off += (size_t)kSmallMats * R * R * 4 + 3 * 32 * 4 + 64;
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
  float* red;   // 32 reduction slots
  int* ibuf;    // 16 ints
};

// out(o, t) = sum_q U(o, q) in(q, t), U = core (nI x nJ) or its transpose.
// Threads are laid out as (chunk, row): the inner index range is split in nch
// chunks whose partial sums are added in a fixed order (deterministic).
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
    if (transposed) {
      for (int q = q0; q < q1; ++q) {
        const float u = U[(size_t)q * ldu + o];
        const float* m = in + (size_t)q * rx;
#pragma unroll
        for (int t = 0; t < R; ++t) acc[t] = fmaf(u, m[t], acc[t]);
      }
    } else {
      for (int q = q0; q < q1; ++q) {
        const float u = U[(size_t)o * ldu + q];
        const float* m = in + (size_t)q * rx;
#pragma unroll
        for (int t = 0; t < R; ++t) acc[t] = fmaf(u, m[t], acc[t]);
      }
    }
    if (nch == 1) {
#pragma unroll
      for (int t = 0; t < R; ++t) out[(size_t)o * rx + t] = acc[t];
    } else {
#pragma unroll
      for (int t = 0; t < R; ++t) part[((size_t)c * rows32 + o) * rx + t] = acc[t];
    }
  }
  __syncthreads();
  if (nch > 1) {
    for (int idx = threadIdx.x; idx < nout * R; idx += blockDim.x) {
      const int oo = idx / R, t = idx % R;
      float s = 0.f;
      for (int cc = 0; cc < nch; ++cc) s += part[((size_t)cc * rows32 + oo) * rx + t];
      out[(size_t)oo * rx + t] = s;
    }
    __syncthreads();
  }
}

template <int R>
__device__ __forceinline__ float sel(const float (&g)[R], int t) {
  float v = 0.f;
#pragma unroll
  for (int u = 0; u < R; ++u)
    if (u == t) v = g[u];
  return v;
}

// Cholesky QR of the nrows x r block Min (stride rx) into Mout (may alias):
// Min = Mout U with U upper triangular (written to Uout).  The Gram matrix is
// formed by warps (one entry per warp), factorised by warp 0 (lane l holds row
// l of the Schur complement), and applied by forward substitution row by row.
// Pivots <= 1e-12 of the largest diagonal entry mark dependent columns: they
// become zero columns and are counted (returned).
template <int R>
__device__ int cholqr(const float* Min, float* Mout, int nrows, int r, int rx, float* Uout, const SvdSmall& sm) {
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
    for (int i = lane; i < nrows; i += 32) acc = fmaf(Min[(size_t)i * rx + s], Min[(size_t)i * rx + t], acc);
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
      const float gt = sel<R>(g, t);  // this lane's entry (lane, t) = (t, lane) of the complement
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
    for (int s = 0; s < R; ++s) m[s] = Min[(size_t)i * rx + s];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      float v = m[t];
#pragma unroll
      for (int s = 0; s < t; ++s) v = fmaf(-y[s], Uout[s * R + t], v);
      y[t] = v * sm.dinv[t];
    }
#pragma unroll
    for (int t = 0; t < R; ++t) Mout[(size_t)i * rx + t] = y[t];
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

template <int R>
__global__ void __launch_bounds__(kSvdThreads, 1) svd_kernel(IterDesc d, int core_in_smem) {
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
  float* Q = reinterpret_cast<float*>(smem + L.off_q);
  float* part = reinterpret_cast<float*>(smem + L.off_part);
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
    p += 32;
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
  int brk = cholqr<R>(X, X, nJ, r, rx, sm.U, sm);
  if (brk > 0) {  // first iteration (B_0 = 0) or a deficient factor: random start
    for (int q = threadIdx.x; q < nJ * rx; q += blockDim.x) {
      const int t = q % rx;
      X[q] = (t < r) ? hash_uniform(d.seed ^ 0x5bd1e995ull, ((uint64_t)k << 32) ^ (uint64_t)q) : 0.f;
    }
    __syncthreads();
    cholqr<R>(X, X, nJ, r, rx, sm.U, sm);
  }

  // ---- subspace iteration
  int steps = 0;
  bool converged = false;
  float prev_res = 0.f;
  while (true) {
    ++steps;
    core_product<R>(Us, ldu, false, nI, nJ, X, Y, part, rx);  // Y = core X
    cholqr<R>(Y, Y, nI, r, rx, sm.Rp, sm);                     // Y Rp = core X
    core_product<R>(Us, ldu, true, nJ, nI, Y, Q, part, rx);    // Q = core^T Y
    // ||Q - X Rp^T||_F^2 and ||Rp||_F^2 in one block reduction
    float e2 = 0.f;
    for (int q = threadIdx.x; q < nJ * r; q += blockDim.x) {
      const int b = q / r, t = q - b * r;
      float v = Q[(size_t)b * rx + t];
      for (int s = t; s < r; ++s) v = fmaf(-X[(size_t)b * rx + s], sm.Rp[t * R + s], v);
      e2 = fmaf(v, v, e2);
    }
    float rc2 = 0.f;
    if (threadIdx.x < R * R) rc2 = sm.Rp[threadIdx.x] * sm.Rp[threadIdx.x];
    e2 = warp_sum(e2);
    rc2 = warp_sum(rc2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      sm.red[warp] = e2;
      sm.red[16 + warp] = rc2;
    }
    __syncthreads();
    float E2 = 0.f, RC2 = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      E2 += sm.red[w];
      RC2 += sm.red[16 + w];
    }
    const float res = sqrtf(E2), nrm = sqrtf(RC2);
    if (res <= 1e-6f * nrm || (steps > 1 && res > 0.5f * prev_res && res <= 1e-5f * nrm) || !(nrm > 0.f)) {
      converged = true;
      break;
    }
    if (steps >= d.svdMaxSteps) break;  // keep X, Y, Rp of the same step
    prev_res = res;
    cholqr<R>(Q, X, nJ, r, rx, sm.U, sm);  // X = orth(core^T Y)
  }

  // ---- second CholQR passes; T = U2y Rp U2x^{-1} = Y^T core X for the new bases
  cholqr<R>(Y, Y, nI, r, rx, sm.U2y, sm);
  cholqr<R>(X, X, nJ, r, rx, sm.U2x, sm);
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
            const float c = rsqrtf(1.f + tt * tt), s = c * tt;
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
    __syncwarp();
    if (p == 0) {
      const float s0 = sm.sig[0];
      const float tol = (float)(nI > nJ ? nI : nJ) * FLT_EPSILON * s0;
      int rank = 0;
      for (int t = 0; t < r; ++t) rank += sm.sig[t] > tol && sm.sig[t] > 0.f;
      sm.ibuf[1] = rank;
      for (int t = r; t < R; ++t) sm.sig[t] = 0.f;
    }
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
