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
    case 20: return launch_recon_r<20>(A, B, n1, n2, D, ldD, L, ldL, S, ldS, st, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// CUR factors of the last iterate K (Alg. 1 output "C_k, U_k, R_k"), on
// request: C = [D - S_K]_{:,J}, R = [D - S_K]_{I,:} recomputed from D with
// the factors and threshold of iteration K-1 (the same FMA chain as the panel
// passes, so the entries are those the solve used), and U = H_r(core) =
// Y T X^T = W V^T from the last core factorisation.
template <int R>
__global__ void __launch_bounds__(256) get_cur_kernel(IterDesc d, int K, const float* __restrict__ D, int64_t ldD,
                                                      float* __restrict__ C, float* __restrict__ U,
                                                      float* __restrict__ Rm) {
  const int prev = (K - 1) & 1;
  const int draw = d.resample ? K - 1 : 0;
  const int* I = d.I_all + (int64_t)draw * d.nI;
  const int* J = d.J_all + (int64_t)draw * d.nJ;
  const float zeta = (float)d.st->zeta_last;
  const float* A = d.A[prev];
  const float* B = d.B[prev];
  const int64_t nC = d.n1 * d.nJ, nR = (int64_t)d.nI * d.n2, nU = (int64_t)d.nI * d.nJ;
  const int64_t total = (C ? nC : 0) + (Rm ? nR : 0) + (U ? nU : 0);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = q;
    if (C && e < nC) {
      const int64_t i = e / d.nJ;
      const int b = (int)(e - i * d.nJ);
      const int64_t j = J[b];
      float arow[R], bcol[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        arow[t] = A[i * R + t];
        bcol[t] = B[(int64_t)t * d.n2 + j];
      }
      C[e] = panel_value(D[i * ldD + j], lowrank_entry<R>(arow, bcol), zeta);
      continue;
    }
    if (C) e -= nC;
    if (Rm && e < nR) {
      const int a = (int)(e / d.n2);
      const int64_t j = e - (int64_t)a * d.n2;
      const int64_t i = I[a];
      float arow[R], bcol[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        arow[t] = A[i * R + t];
        bcol[t] = B[(int64_t)t * d.n2 + j];
      }
      Rm[e] = panel_value(D[i * ldD + j], lowrank_entry<R>(arow, bcol), zeta);
      continue;
    }
    if (Rm) e -= nR;
    const int a = (int)(e / d.nJ);
    const int b = (int)(e - (int64_t)a * d.nJ);
    float u = 0.f;
#pragma unroll
    for (int t = 0; t < R; ++t) u = fmaf(d.W[(size_t)a * R + t], d.V[(size_t)b * R + t], u);
    U[e] = u;
  }
}

cudaError_t launch_get_cur(const IterDesc& d, int Rpad, int K, const float* D, int64_t ldD, float* C, float* U,
                           float* Rm, cudaStream_t s) {
  const int blocks = 4 * kNumSMsHint;
  switch (Rpad) {
#define IRCUR_CUR_CASE(RR) \
  case RR:                 \
    get_cur_kernel<RR><<<blocks, 256, 0, s>>>(d, K, D, ldD, C, U, Rm); \
    break;
    IRCUR_CUR_CASE(1)
    IRCUR_CUR_CASE(2)
    IRCUR_CUR_CASE(3)
    IRCUR_CUR_CASE(4)
    IRCUR_CUR_CASE(5)
    IRCUR_CUR_CASE(6)
    IRCUR_CUR_CASE(7)
    IRCUR_CUR_CASE(8)
    IRCUR_CUR_CASE(9)
    IRCUR_CUR_CASE(10)
    IRCUR_CUR_CASE(12)
    IRCUR_CUR_CASE(16)
    IRCUR_CUR_CASE(20)
#undef IRCUR_CUR_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ircur
