// Solve set-up kernels: index sampling (Alg. 1, uniform I and J), index-set
// validation, max|D| for zeta_0 (Sec. 3.5), the fixed-index panel gathers of
// IRCUR-F (Sec. 3.4) and the state reset.
#include <float.h>

#include "device_common.cuh"
#include "ircur_internal.cuh"
#include "sampler.cuh"

namespace ircur {

// ---------------------------------------------------------------------------
// Index sets for `draws` consecutive draws (blockIdx.x) and one or both axes
// (blockIdx.y), one block per set; see sampler.cuh.
__global__ void __launch_bounds__(1024) sample_kernel(uint64_t seed, int draw0, int64_t n1, int64_t n2,
                                                      int nI, int nJ, int* I_all, int* J_all, int only_axis,
                                                      unsigned* mapI0, unsigned* mapI1, unsigned* mapJ0,
                                                      unsigned* mapJ1) {
  __shared__ SamplerSmem S;
  const int axis = only_axis >= 0 ? only_axis : (int)blockIdx.y;
  const int draw = draw0 + (int)blockIdx.x;
  int* out = axis ? (J_all + (int64_t)blockIdx.x * nJ) : (I_all + (int64_t)blockIdx.x * nI);
  unsigned* map = axis ? ((draw & 1) ? mapJ1 : mapJ0) : ((draw & 1) ? mapI1 : mapI0);
  sample_subset(seed, draw, axis, axis ? n2 : n1, axis ? nJ : nI, out, S, map, (unsigned)(draw + 1));
}

cudaError_t launch_sample(uint64_t seed, int draw0, int draws, int64_t n1, int64_t n2, int nI, int nJ,
                          int* I_all, int* J_all, int only_axis, cudaStream_t s, unsigned* const* mapI,
                          unsigned* const* mapJ) {
  dim3 grid(draws, only_axis >= 0 ? 1 : 2);
  sample_kernel<<<grid, 1024, 0, s>>>(seed, draw0, n1, n2, nI, nJ, I_all, J_all, only_axis,
                                      mapI ? mapI[0] : nullptr, mapI ? mapI[1] : nullptr,
                                      mapJ ? mapJ[0] : nullptr, mapJ ? mapJ[1] : nullptr);
  return cudaGetLastError();
}

// The index maps of caller-supplied sets: map[idx[a]] = index_tag(draw + 1, a).
// Runs after their check; sets that failed it are never dereferenced.
__global__ void index_map_kernel(const int* __restrict__ idx, int m, unsigned* __restrict__ map, unsigned tag,
                                 const State* st) {
  if (st->status) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < m; a += gridDim.x * blockDim.x)
    map[idx[a]] = index_tag(tag, a);
}

cudaError_t launch_index_map(const int* idx, int m, unsigned* map, int draw, const State* st, cudaStream_t s) {
  index_map_kernel<<<(m + 255) / 256, 256, 0, s>>>(idx, m, map, (unsigned)(draw + 1), st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Caller-supplied index sets: strictly ascending, inside [0, n).
__global__ void check_indices_kernel(const int* idx, int sets, int m, int64_t n, int* status) {
  const int64_t total = (int64_t)sets * m;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(q % m);
    const int v = idx[q];
    bool bad = v < 0 || (int64_t)v >= n;
    if (p > 0 && idx[q - 1] >= v) bad = true;
    if (bad) atomicExch(status, (int)IRCUR_EINVAL);
  }
}

cudaError_t launch_check_indices(const int* idx, int sets, int m, int64_t n, int* status,
                                 cudaStream_t s) {
  const int64_t total = (int64_t)sets * m;
  int blocks = (int)((total + 255) / 256);
  blocks = blocks < 1 ? 1 : (blocks > 4 * kNumSMsHint ? 4 * kNumSMsHint : blocks);
  check_indices_kernel<<<blocks, 256, 0, s>>>(idx, sets, m, n, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// max|D_ij| over the whole matrix (zeta_0 = max|D| reading) and a NaN/Inf scan.
// Streaming read of D: 16-byte loads when rows are 16-byte aligned.
__global__ void __launch_bounds__(256) maxabs_kernel(const float* __restrict__ D, int64_t n1,
                                                     int64_t n2, int64_t ldD, int vec,
                                                     State* st) {
  float m = 0.f;
  bool bad = false;
  if (vec) {
    const int64_t n4 = n2 >> 2;
    for (int64_t i = blockIdx.x; i < n1; i += gridDim.x) {
      const float4* row = reinterpret_cast<const float4*>(D + i * ldD);
      int64_t j = threadIdx.x;
      for (; j + 3 * 256 < n4; j += 4 * 256) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = __ldcs(row + j + u * 256);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float a = fmaxf(fmaxf(fabsf(v[u].x), fabsf(v[u].y)), fmaxf(fabsf(v[u].z), fabsf(v[u].w)));
          bad |= !(fabsf(v[u].x) <= FLT_MAX) || !(fabsf(v[u].y) <= FLT_MAX) ||
                 !(fabsf(v[u].z) <= FLT_MAX) || !(fabsf(v[u].w) <= FLT_MAX);
          m = fmaxf(m, a);
        }
      }
      for (; j < n4; j += 256) {
        const float4 v = __ldcs(row + j);
        bad |= !(fabsf(v.x) <= FLT_MAX) || !(fabsf(v.y) <= FLT_MAX) || !(fabsf(v.z) <= FLT_MAX) ||
               !(fabsf(v.w) <= FLT_MAX);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
      }
      for (int64_t jj = (n4 << 2) + threadIdx.x; jj < n2; jj += 256) {
        const float x = D[i * ldD + jj];
        bad |= !(fabsf(x) <= FLT_MAX);
        m = fmaxf(m, fabsf(x));
      }
    }
  } else {
    for (int64_t i = blockIdx.x; i < n1; i += gridDim.x)
      for (int64_t j = threadIdx.x; j < n2; j += 256) {
        const float x = D[i * ldD + j];
        bad |= !(fabsf(x) <= FLT_MAX);
        m = fmaxf(m, fabsf(x));
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  bad = __any_sync(0xffffffffu, bad);
  __shared__ float wm[8];
  __shared__ int wb[8];
  if ((threadIdx.x & 31) == 0) {
    wm[threadIdx.x >> 5] = m;
    wb[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    int anybad = 0;
    for (int w = 0; w < 8; ++w) {
      b = fmaxf(b, wm[w]);
      anybad |= wb[w];
    }
    atomicMax(&st->maxabs_bits, __float_as_uint(b));
    if (anybad) atomicExch(&st->nonfinite, 1);
  }
}

__global__ void finalize_zeta_kernel(State* st) {
  if (st->nonfinite) {
    st->status = IRCUR_EINVAL;
    st->done = 1;
    return;
  }
  const double z = (double)__uint_as_float(st->maxabs_bits);
  st->zeta0 = z;
  st->zeta = z;
}

cudaError_t launch_maxabs(const float* D, int64_t n1, int64_t n2, int64_t ldD, State* st,
                          cudaStream_t s) {
  const int vec = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && (ldD % 4 == 0);
  int blocks = (int)(n1 < 8 * kNumSMsHint ? n1 : 8 * kNumSMsHint);
  if (blocks < 1) blocks = 1;
  maxabs_kernel<<<blocks, 256, 0, s>>>(D, n1, n2, ldD, vec, st);
  return cudaGetLastError();
}

cudaError_t launch_finalize_zeta(State* st, cudaStream_t s) {
  finalize_zeta_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// IRCUR-R: D^T (n2 x n1) once per solve, so that the column panels D(:,J_k)
// of every iteration are row gathers of D^T; the same pass takes max|D| and
// the NaN/Inf scan.  64 x 64 tiles through padded shared memory, 256 threads:
// 16-byte streaming loads along rows of D (when rows are 16-byte aligned),
// 16-byte stores along rows of D^T, all coalesced.
constexpr int kTT = 64;
__global__ void __launch_bounds__(256) transpose_maxabs_kernel(const float* __restrict__ D, int64_t n1,
                                                               int64_t n2, int64_t ldD, float* __restrict__ DT,
                                                               int64_t ldDT, int vec, State* st) {
  __shared__ float tile[kTT][kTT + 1];
  const int64_t tiles_i = (n1 + kTT - 1) / kTT, tiles_j = (n2 + kTT - 1) / kTT;
  const int64_t ntiles = tiles_i * tiles_j;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16
  float m = 0.f;
  bool bad = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t ti = t / tiles_j, tj = t - ti * tiles_j;
    const int64_t i0 = ti * kTT, j0 = tj * kTT;
    const bool full = vec && i0 + kTT <= n1 && j0 + kTT <= n2;
    if (full) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = __ldcs(reinterpret_cast<const float4*>(D + (i0 + ty + 16 * q) * ldD + j0) + tx);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float e[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          bad |= !(fabsf(e[u]) <= FLT_MAX);
          m = fmaxf(m, fabsf(e[u]));
          tile[ty + 16 * q][4 * tx + u] = e[u];
        }
      }
    } else {
      for (int q = threadIdx.x; q < kTT * kTT; q += blockDim.x) {
        const int r = q / kTT, cc = q - r * kTT;
        const int64_t i = i0 + r, j = j0 + cc;
        float x = 0.f;
        if (i < n1 && j < n2) {
          x = D[i * ldD + j];
          bad |= !(fabsf(x) <= FLT_MAX);
          m = fmaxf(m, fabsf(x));
        }
        tile[r][cc] = x;
      }
    }
    __syncthreads();
    if (full) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int jr = ty + 16 * q;  // row of D^T inside the tile
        float4 o;
        o.x = tile[4 * tx + 0][jr];
        o.y = tile[4 * tx + 1][jr];
        o.z = tile[4 * tx + 2][jr];
        o.w = tile[4 * tx + 3][jr];
        reinterpret_cast<float4*>(DT + (j0 + jr) * ldDT + i0)[tx] = o;
      }
    } else {
      for (int q = threadIdx.x; q < kTT * kTT; q += blockDim.x) {
        const int jr = q / kTT, ic = q - jr * kTT;
        const int64_t j = j0 + jr, i = i0 + ic;
        if (i < n1 && j < n2) DT[j * ldDT + i] = tile[ic][jr];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  bad = __any_sync(0xffffffffu, bad);
  __shared__ float wm[8];
  __shared__ int wb[8];
  if ((threadIdx.x & 31) == 0) {
    wm[threadIdx.x >> 5] = m;
    wb[threadIdx.x >> 5] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    int anybad = 0;
    for (int w = 0; w < 8; ++w) {
      b = fmaxf(b, wm[w]);
      anybad |= wb[w];
    }
    atomicMax(&st->maxabs_bits, __float_as_uint(b));
    if (anybad) atomicExch(&st->nonfinite, 1);
  }
}

cudaError_t launch_transpose_maxabs(const float* D, int64_t n1, int64_t n2, int64_t ldD, float* DT,
                                    int64_t ldDT, State* st, cudaStream_t s) {
  const int64_t ntiles = ((n1 + kTT - 1) / kTT) * ((n2 + kTT - 1) / kTT);
  int blocks = (int)(ntiles < 8 * kNumSMsHint ? ntiles : 8 * kNumSMsHint);
  if (blocks < 1) blocks = 1;
  const int vec = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && (ldD % 4 == 0) &&
                  ((reinterpret_cast<uintptr_t>(DT) & 15) == 0) && (ldDT % 4 == 0);
  transpose_maxabs_kernel<<<blocks, 256, 0, s>>>(D, n1, n2, ldD, DT, ldDT, vec, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State reset at the start of a solve.
__global__ void setup_kernel(State* st, double zeta0, int max_iter) {
  st->k = 0;
  st->done = max_iter <= 0;
  st->status = 0;
  st->flags = 0u;
  st->zeta = zeta0;
  st->zeta0 = zeta0;
  st->e = 1.0;
  st->counter = 0u;
  st->maxabs_bits = 0u;
  st->nonfinite = 0;
  st->svd_steps = 0;
  st->svd_last_steps = 0;
}

cudaError_t launch_setup(const IterDesc& d, double zeta0, cudaStream_t s) {
  setup_kernel<<<1, 1, 0, s>>>(d.st, zeta0, d.max_iter);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// IRCUR-F: gather the fixed panels once, D(I,:) -> Prow (nI x ldPr) and
// D(:,J)^T -> PcolT (nJ x ldPc, row b holds column J_b of D).
__global__ void __launch_bounds__(256) gather_rows_kernel(IterDesc d) {
  if (d.st->status) return;  // caller index sets that failed their check are never dereferenced
  const int a = blockIdx.y;
  const float* src = d.D + (int64_t)d.I_all[a] * d.ldD;
  if (d.bf16) {
    uint16_t* dst = const_cast<uint16_t*>(d.rowSrcH) + (int64_t)a * d.rowLd;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n2; j += (int64_t)gridDim.x * blockDim.x)
      dst[j] = f32_to_bf16_bits(__ldg(src + j));
    return;
  }
  float* dst = d.Prow + (int64_t)a * d.ldPr;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < d.n2;
       j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = __ldg(src + j);
}

__global__ void __launch_bounds__(256) gather_cols_kernel(IterDesc d) {
  if (d.st->status) return;
  const int b = blockIdx.y;
  const int64_t j = d.J_all[b];
  if (d.bf16) {
    uint16_t* dst = const_cast<uint16_t*>(d.colSrcH) + (int64_t)b * d.colLd;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n1; i += (int64_t)gridDim.x * blockDim.x)
      dst[i] = f32_to_bf16_bits(__ldg(d.D + i * d.ldD + j));
    return;
  }
  float* dst = d.PcolT + (int64_t)b * d.ldPc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d.n1;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __ldg(d.D + i * d.ldD + j);
}

cudaError_t launch_gather(const IterDesc& d, cudaStream_t s) {
  int gx = (int)((d.n2 + 255) / 256);
  if (gx > 64) gx = 64;
  gather_rows_kernel<<<dim3(gx, d.nI), 256, 0, s>>>(d);
  int gy = (int)((d.n1 + 255) / 256);
  if (gy > 64) gy = 64;
  gather_cols_kernel<<<dim3(gy, d.nJ), 256, 0, s>>>(d);
  return cudaGetLastError();
}

}  // namespace ircur

namespace ircur {

// ---------------------------------------------------------------------------
// D(I,J) of one draw into the compact buffer the core SVD reads, Dc[buf]
// (nI x ldDc).  IRCUR-F
// gathers it once per solve; IRCUR-R gathers draw 0 here and every later draw
// in the previous iteration's panel pass.
__global__ void __launch_bounds__(256) gather_core_kernel(IterDesc d, int draw, int buf) {
  if (d.st->status) return;  // caller index sets that failed their check are never dereferenced
  const int* I = d.I_all + (int64_t)draw * d.nI;
  const int* J = d.J_all + (int64_t)draw * d.nJ;
  const int64_t total = (int64_t)d.nI * d.nJ;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / d.nJ), b = (int)(e - (int64_t)a * d.nJ);
    const float v = __ldg(d.D + (int64_t)I[a] * d.ldD + J[b]);
    d.Dc[buf][(int64_t)a * d.ldDc + b] = v;
  }
}

cudaError_t launch_gather_core(const IterDesc& d, int draw, int buf, cudaStream_t s) {
  const int64_t total = (int64_t)d.nI * d.nJ;
  int blocks = (int)((total + 255) / 256);
  blocks = blocks < 1 ? 1 : (blocks > 4 * kNumSMsHint ? 4 * kNumSMsHint : blocks);
  gather_core_kernel<<<blocks, 256, 0, s>>>(d, draw, buf);
  return cudaGetLastError();
}

}  // namespace ircur
