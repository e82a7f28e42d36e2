// Dense output of the final iterate: L = C U^+ R = A B (Thm 1 with the
// factorisation A = C V_r Sigma_r^{-1}, B = W_r^T R) and optionally the
// sparse part S = T_zeta(D - L) (Sec. 3.2, strict >) at zeta = gamma^K zeta_0.
//
// The contraction has K = r <= 16, i.e. 2r flops per 4 (L only) or 12 (L and
// S) bytes of HBM traffic: the kernel is bound by HBM writes, not by any
// arithmetic pipe, so it runs on CUDA-core FMAs with 16-byte streaming
// stores.  Each thread owns 4 consecutive columns and keeps their B values in
// registers across a run of rows; A rows are broadcast loads.
#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

constexpr int kReconThreads = 256;
constexpr int kReconRows = 16;  // rows per block

template <int R, bool WITH_S>
__global__ void __launch_bounds__(kReconThreads) recon_vec_kernel(const float* __restrict__ A,
                                                                 const float* __restrict__ B, int64_t n1,
                                                                 int64_t n2, const float* __restrict__ D,
                                                                 int64_t ldD, float* __restrict__ L,
                                                                 int64_t ldL, float* __restrict__ S,
                                                                 int64_t ldS, const State* st) {
  const float zeta = WITH_S ? (float)st->zeta : 0.f;
  const int64_t j = ((int64_t)blockIdx.x * kReconThreads + threadIdx.x) * 4;
  if (j >= n2) return;
  const int64_t i0 = (int64_t)blockIdx.y * kReconRows;
  const int64_t i1 = i0 + kReconRows < n1 ? i0 + kReconRows : n1;
  const bool full = j + 3 < n2;
  float4 b[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const float* bp = B + (int64_t)t * n2 + j;
    if (full) {
      b[t] = make_float4(bp[0], bp[1], bp[2], bp[3]);
    } else {
      b[t].x = bp[0];
      b[t].y = j + 1 < n2 ? bp[1] : 0.f;
      b[t].z = j + 2 < n2 ? bp[2] : 0.f;
      b[t].w = 0.f;
    }
  }
  for (int64_t i = i0; i < i1; ++i) {
    float a[R];
#pragma unroll
    for (int t = 0; t < R; ++t) a[t] = __ldg(A + i * R + t);
    float4 l = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      l.x = fmaf(a[t], b[t].x, l.x);
      l.y = fmaf(a[t], b[t].y, l.y);
      l.z = fmaf(a[t], b[t].z, l.z);
      l.w = fmaf(a[t], b[t].w, l.w);
    }
    if (full) {
      st_stream(reinterpret_cast<float4*>(L + i * ldL + j), l);
      if (WITH_S) {
        const float4 dv = __ldcs(reinterpret_cast<const float4*>(D + i * ldD + j));
        float4 s;
        s.x = fabsf(dv.x - l.x) > zeta ? dv.x - l.x : 0.f;
        s.y = fabsf(dv.y - l.y) > zeta ? dv.y - l.y : 0.f;
        s.z = fabsf(dv.z - l.z) > zeta ? dv.z - l.z : 0.f;
        s.w = fabsf(dv.w - l.w) > zeta ? dv.w - l.w : 0.f;
        st_stream(reinterpret_cast<float4*>(S + i * ldS + j), s);
      }
    } else {
      const float lv[4] = {l.x, l.y, l.z, l.w};
      for (int c = 0; c < 4 && j + c < n2; ++c) {
        L[i * ldL + j + c] = lv[c];
        if (WITH_S) {
          const float res = D[i * ldD + j + c] - lv[c];
          S[i * ldS + j + c] = fabsf(res) > zeta ? res : 0.f;
        }
      }
    }
  }
}

// Scalar variant for buffers that are not 16-byte aligned row by row.
template <int R, bool WITH_S>
__global__ void __launch_bounds__(kReconThreads) recon_scalar_kernel(const float* __restrict__ A,
                                                                    const float* __restrict__ B, int64_t n1,
                                                                    int64_t n2, const float* __restrict__ D,
                                                                    int64_t ldD, float* __restrict__ L,
                                                                    int64_t ldL, float* __restrict__ S,
                                                                    int64_t ldS, const State* st) {
  const float zeta = WITH_S ? (float)st->zeta : 0.f;
  const int64_t j = (int64_t)blockIdx.x * kReconThreads + threadIdx.x;
  if (j >= n2) return;
  float b[R];
#pragma unroll
  for (int t = 0; t < R; ++t) b[t] = B[(int64_t)t * n2 + j];
  const int64_t i0 = (int64_t)blockIdx.y * kReconRows;
  const int64_t i1 = i0 + kReconRows < n1 ? i0 + kReconRows : n1;
  for (int64_t i = i0; i < i1; ++i) {
    float l = 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) l = fmaf(__ldg(A + i * R + t), b[t], l);
    L[i * ldL + j] = l;
    if (WITH_S) {
      const float res = D[i * ldD + j] - l;
      S[i * ldS + j] = fabsf(res) > zeta ? res : 0.f;
    }
  }
}

template <int R>
static cudaError_t launch_recon_r(const float* A, const float* B, int64_t n1, int64_t n2, const float* D,
                                  int64_t ldD, float* L, int64_t ldL, float* S, int64_t ldS,
                                  const State* st, cudaStream_t s) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const bool vec = al16(L) && ldL % 4 == 0 && (!S || (al16(S) && ldS % 4 == 0 && al16(D) && ldD % 4 == 0));
  const unsigned gy = (unsigned)((n1 + kReconRows - 1) / kReconRows);
  if (vec) {
    const unsigned gx = (unsigned)((n2 + 4 * kReconThreads - 1) / (4 * kReconThreads));
    if (S)
      recon_vec_kernel<R, true><<<dim3(gx, gy), kReconThreads, 0, s>>>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st);
    else
      recon_vec_kernel<R, false><<<dim3(gx, gy), kReconThreads, 0, s>>>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st);
  } else {
    const unsigned gx = (unsigned)((n2 + kReconThreads - 1) / kReconThreads);
    if (S)
      recon_scalar_kernel<R, true><<<dim3(gx, gy), kReconThreads, 0, s>>>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st);
    else
      recon_scalar_kernel<R, false><<<dim3(gx, gy), kReconThreads, 0, s>>>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_reconstruct(const float* A, const float* B, int Rpad, int64_t n1, int64_t n2,
                               const float* D, int64_t ldD, float* L, int64_t ldL, float* S, int64_t ldS,
                               const State* st, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_recon_r<1>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 2: return launch_recon_r<2>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 3: return launch_recon_r<3>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 4: return launch_recon_r<4>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 5: return launch_recon_r<5>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 6: return launch_recon_r<6>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 7: return launch_recon_r<7>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 8: return launch_recon_r<8>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 9: return launch_recon_r<9>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 10: return launch_recon_r<10>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 12: return launch_recon_r<12>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    case 16: return launch_recon_r<16>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ircur
