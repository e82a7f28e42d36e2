// One IRCUR iteration (Alg. 1) on the GPU, in two kernels:
//   svd_kernel   -- [D - S_{k+1}]_{I,J} (Phase I on the |I| x |J| block), H_r
//                   of that core and its pseudo-inverse (k_svd.cu),
//   pass_kernel  -- the fused row- and column-panel passes and the stopping
//                   criterion.
//
// The iterate L_k = C_k U_k^+ R_k is never formed (Alg. 1); it is carried as
// the skinny factors A_k = C_k V_r Sigma_r^{-1} (n1 x r) and B_k = W_r^T R_k
// (r x n2), L_k = A_k B_k, so [L_k]_{I,:} and [L_k]_{:,J} (the two panel
// formulas of Sec. 3.2) are evaluated entry by entry as A_k(i,:) B_k(:,j).
// With U = W_r Sigma_r V_r^T the update C U^+ R factors as
// (C V_r Sigma_r^{-1})(W_r^T R): the column pass produces A_{k+1}, the row
// pass B_{k+1}.  Because C(I,:) = R(:,J) = core, L_{k+1}(I,:) = W_r W_r^T R
// and L_{k+1}(:,J) = C V_r V_r^T, so the stopping criterion of Sec. 3.3 is
// e = (||R - W_r W_r^T R||_F + ||C - C V_r V_r^T||_F) / (||D_{I,:}||_F + ||D_{:,J}||_F),
// each residual formed explicitly (no difference of squared norms).
#include <string.h>

#include <mutex>

#include "device_common.cuh"
#include "ircur_internal.cuh"

namespace ircur {

int pad_rank(int r) {
  if (r <= 10) return r;
  if (r <= 12) return 12;
  if (r <= 16) return 16;
  return 20;
}

// ---------------------------------------------------------------------------
// Panel passes: Alg. 1 Phase I on the panels, the Phase II products and the
// stopping sums of Sec. 3.3, as one persistent grid over tiles of kPanelCols
// consecutive panel columns.
//
// Row pass (COL = false): the panel is D(I,:) (m = |I| rows); for column j
//   R_{k+1}(:,j) = D(I,j) - T_zeta(D(I,j) - A_k(I,:) B_k(:,j)),
//   B_{k+1}(:,j) = Y^T R_{k+1}(:,j),
//   num += ||R_{k+1}(:,j) - Y B_{k+1}(:,j)||^2,  den += ||D(I,j)||^2.
// Column pass (COL = true): the panel is D(:,J)^T (m = |J| rows); for row i
//   C_{k+1}(i,:) = D(i,J) - T_zeta(D(i,J) - A_k(i,:) B_k(:,J)),
//   A_{k+1}(i,:) = C_{k+1}(i,:) X T^{-1},
//   num += ||C_{k+1}(i,:) - A_{k+1}(i,:) T X^T||^2,  den += ||D(i,J)||^2.
// Both are the same computation on a row-major m x n panel with
//   side = A_k(I,:) | B_k(:,J)^T (m x R), vec = B_k(:,j) | A_k(i,:)^T,
//   proj = Y | X T^{-1},  recon = Y | X T^T  (U^+ = X T^{-1} Y^T, see k_svd.cu).
//
// A block owns a contiguous run of tiles (the grid is the number of resident
// blocks); consecutive tiles of one instance and side form a segment whose
// m x R side, projection and reconstruction matrices are staged in shared
// memory once.  The kernel is launched as a programmatic dependent of the core
// SVD: its blocks start while the SVD (one cluster) runs, stage and threshold
// their first tile, and wait for the SVD only before the projections.  Tiles are double-buffered: the 16-byte asynchronous copies of
// tile t+1 (one small segment per gathered panel row) fly while tile t is
// computed.  Within a tile, warp h owns row share h and lane c column c
// (conflict-free tile accesses, broadcast reads of the small matrices); the
// share partial projections and the shares' num/den sums are added in a fixed
// order into one slot per tile, so e_{k+1} does not depend on how the tiles
// are spread over blocks.  The block that completes an
// instance's last tile reduces its slots in a fixed order, evaluates e_{k+1},
// advances k and zeta, and (single instance) drives the graph's while-node
// (Alg. 1: "while e_k > epsilon").

struct PassLayout {
  int m, rx, nbuf;
  unsigned char* tiles;  // nbuf staging buffers of m x kPanelCols panel entries (FP32 or BF16)
  size_t tile_bytes;     // bytes of one staging buffer
  float* vbuf;           // BF16 panels: the FP32 values D - S of the current tile (else null)
  float* side;
  float* proj;
  float* recon;
  float* part;  // nw x RX x kPanelCols (nw: warps of the block)
  float* outS;  // RX x kPanelCols
  float* wsum;  // nw x 2
  float* lvec;      // nbuf x (kPanelCols x RX): the tile's columns of the other factor (pass_stage_lane)
  unsigned* lpos;   // nbuf x kPanelCols: the next draw's position-map entries of the tile's columns
  int* idx;         // 2 m: I_k then J_k (IRCUR-R, single instance), the rows the tiles gather
};

__host__ __device__ inline size_t pass_layout_floats(int m, int rx, int nbuf, bool bf16, int nw) {
  const size_t tile = bf16 ? (size_t)m * kPanelCols / 2 : (size_t)m * kPanelCols;  // in floats
  return (size_t)nbuf * tile + (bf16 ? (size_t)m * kPanelCols : 0) + 3 * (size_t)m * rx +
         (size_t)nw * rx * kPanelCols + (size_t)rx * kPanelCols + 4 * nw +
         (size_t)nbuf * ((size_t)kPanelCols * rx + kPanelCols) + 2 * (size_t)m;
}

__device__ inline PassLayout pass_layout(unsigned char* smem, int m, int rx, int nbuf, bool bf16, int nw) {
  PassLayout L;
  L.m = m;
  L.rx = rx;
  L.nbuf = nbuf;
  L.tiles = smem;
  // m is a multiple of... any m: round the BF16 buffers to 16 bytes
  L.tile_bytes = bf16 ? (((size_t)m * kPanelCols * 2 + 15) & ~(size_t)15) : (size_t)m * kPanelCols * 4;
  float* p = reinterpret_cast<float*>(smem + nbuf * L.tile_bytes);
  L.vbuf = bf16 ? p : nullptr;
  if (bf16) p += (size_t)m * kPanelCols;
  L.side = p;
  L.proj = p + (size_t)m * rx;
  L.recon = p + 2 * (size_t)m * rx;
  L.part = p + 3 * (size_t)m * rx;
  L.outS = L.part + (size_t)nw * rx * kPanelCols;
  L.wsum = L.outS + (size_t)rx * kPanelCols;
  L.lvec = L.wsum + 4 * nw;  // 16-byte aligned: every piece above is a multiple of 4 floats
  L.lpos = reinterpret_cast<unsigned*>(L.lvec + (size_t)nbuf * kPanelCols * rx);
  L.idx = reinterpret_cast<int*>(L.lpos + (size_t)nbuf * kPanelCols);
  return L;
}

// Where tile t of the grid lives.
struct TileRef {
  int inst;    // instance
  int col;     // 0: row panel, 1: column panel
  int lt;      // tile within that panel
  int active;  // the instance is still iterating
  int k;       // its iteration
};

// Issue the copies of one panel tile into `buf`: 16-byte asynchronous copies
// when the rows are 16-byte aligned (4-byte ones for the last 1..3 columns of
// a ragged last tile), 4-byte ones otherwise (BF16 panels, always aligned:
// plain loads for the ragged tile).
template <bool COL, bool BF>
__device__ __forceinline__ void pass_stage_tile(const IterDesc& d, int k, int lt, unsigned char* bufp,
                                                const int* smap) {
  const int m = COL ? d.nJ : d.nI;
  const int64_t ncolsTotal = COL ? d.n1 : d.n2;
  const int64_t ld = COL ? d.colLd : d.rowLd;
  const int64_t j0 = (int64_t)lt * kPanelCols;
  const int ncols = (int)((ncolsTotal - j0) < kPanelCols ? (ncolsTotal - j0) : kPanelCols);
  if (BF) {
    const uint16_t* src = COL ? d.colSrcH : d.rowSrcH;
    uint16_t* buf = reinterpret_cast<uint16_t*>(bufp);
    if (ncols == kPanelCols) {
      constexpr int kV = kPanelCols / 8;
      for (int q = threadIdx.x; q < m * kV; q += blockDim.x) {
        const int a = q / kV, c8 = q - a * kV;
        cp_async16(buf + (size_t)a * kPanelCols + 8 * c8, src + (int64_t)a * ld + j0 + 8 * c8);
      }
    } else {
      for (int q = threadIdx.x; q < m * kPanelCols; q += blockDim.x) {
        const int a = q / kPanelCols, c = q - a * kPanelCols;
        buf[q] = c < ncols ? src[(int64_t)a * ld + j0 + c] : (uint16_t)0;
      }
    }
    return;
  }
  float* buf = reinterpret_cast<float*>(bufp);
  // the gathered rows: the block's shared copy of the index set, else global
  const int* map = smap ? smap : (COL ? d.J_all : d.I_all) + (d.resample ? (int64_t)k * m : 0);
  const bool mapped = d.resample != 0;
  const float* src = COL ? d.colSrc : d.rowSrc;
  if (COL ? d.colBulk : d.rowBulk) {
    // 16-byte copies of whole 4-column groups; on the ragged last tile the
    // remaining 1..3 columns by 4-byte copies and zeros past the last column
    constexpr int kV = kPanelCols / 4;
    const int nv = ncols >> 2, rem4 = ncols & 3;
    for (int q = threadIdx.x; q < m * kV; q += blockDim.x) {
      const int a = q / kV, c4 = q - a * kV;
      float* dst = buf + (size_t)a * kPanelCols + 4 * c4;
      if (c4 < nv) {
        const int64_t row = mapped ? map[a] : a;
        cp_async16(dst, src + row * ld + j0 + 4 * c4);
      } else if (c4 == nv && rem4) {
        const int64_t row = mapped ? map[a] : a;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (e < rem4)
            cp_async4(dst + e, src + row * ld + j0 + 4 * c4 + e);
          else
            dst[e] = 0.f;
        }
      } else {
        *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  } else {
    // rows not 16-byte aligned: 4-byte asynchronous
    // copies (zeros past the panel's last column)
    for (int q = threadIdx.x; q < m * kPanelCols; q += blockDim.x) {
      const int a = q / kPanelCols, c = q - a * kPanelCols;
      if (c < ncols) {
        const int64_t row = mapped ? map[a] : a;
        cp_async4(buf + q, src + row * ld + j0 + c);
      } else {
        buf[q] = 0.f;
      }
    }
  }
}

// The tile's columns (rows) of the current iterate's other factor, B_k(:,j)
// for the row panel (lv[t kPanelCols + c]) or A_k(i,:) for the column panel
// (lv[c R + t]), and the next draw's position-map entries of the same columns
// (lp[c]), copied asynchronously with the tile; zero past the panel's last
// column.
template <int R, bool COL>
__device__ __forceinline__ void pass_stage_lane(const IterDesc& d, int k, int lt, float* lv, unsigned* lp) {
  const int cur = k & 1;
  const int64_t ncolsTotal = COL ? d.n1 : d.n2;
  const int64_t j0 = (int64_t)lt * kPanelCols;
  const int ncols = (int)((ncolsTotal - j0) < kPanelCols ? (ncolsTotal - j0) : kPanelCols);
  if (COL) {
    // ncols R consecutive floats; the source starts on a 16-byte boundary
    // (j0 R 4 bytes = 128 lt R)
    const float* src = d.A[cur] + j0 * R;
    const int nf = ncols * R, n4 = nf >> 2;
    for (int q = threadIdx.x; q < n4; q += blockDim.x) cp_async16(lv + 4 * q, src + 4 * q);
    for (int q = 4 * n4 + (int)threadIdx.x; q < nf; q += blockDim.x) cp_async4(lv + q, src + q);
    for (int q = nf + (int)threadIdx.x; q < kPanelCols * R; q += blockDim.x) lv[q] = 0.f;
  } else {
    for (int q = threadIdx.x; q < R * kPanelCols; q += blockDim.x) {
      const int t = q / kPanelCols, c = q - t * kPanelCols;
      if (c < ncols)
        cp_async4(lv + q, d.B[cur] + (int64_t)t * d.n2 + j0 + c);
      else
        lv[q] = 0.f;
    }
  }
  const int dnext = d.resample ? k + 1 : 0;
  const unsigned* map = (COL ? d.posI : d.posJ)[dnext & 1] + j0;
  for (int q = threadIdx.x; q < kPanelCols; q += blockDim.x) {
    if (q < ncols)
      cp_async4(lp + q, map + q);
    else
      lp[q] = 0u;
  }
}

// The m x R side matrix of one segment, A_k(I,:) | B_k(:,J)^T: the compact
// copies the previous pass wrote through the index maps (the same values the
// core SVD used for L_k(I,J)), rows padded to RX columns with zeros.
template <int R, bool COL>
__device__ __forceinline__ void pass_stage_side(const IterDesc& d, const PassLayout& L, int k) {
  constexpr int RX = (R + 3) & ~3;
  const int m = COL ? d.nJ : d.nI;
  const float* sideG = COL ? d.BJt[k & 1] : d.AI[k & 1];
  for (int q = threadIdx.x; q < m * RX; q += blockDim.x) {
    const int a = q / RX, t = q - a * RX;
    L.side[q] = t < R ? sideG[(size_t)a * R + t] : 0.f;
  }
}

// IRCUR-R: the core SVD of iteration k + 1 reads D(I_{k+1}, J_{k+1}) from the
// compact buffers [(k + 1) & 1].  Row tile lt of iteration k gathers the core
// rows a = lt, lt + nRowTiles, ... of it before its blocks wait for the core
// SVD (the index sets of k + 1 were drawn an iteration earlier).
__device__ __forceinline__ void pass_gather_next_core(const IterDesc& d, int k, int lt) {
  if (!d.resample || k + 1 >= d.max_iter || lt >= d.nI) return;
  const int rows = (d.nI - 1 - lt) / d.nRowTiles + 1;
  const int total = rows * d.nJ;
  const int* In = d.I_all + (int64_t)(k + 1) * d.nI;
  const int* Jn = d.J_all + (int64_t)(k + 1) * d.nJ;
  const int nb = (k + 1) & 1;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int ra = e / d.nJ, b = e - ra * d.nJ;
    const int a = lt + ra * d.nRowTiles;
    const float v = __ldcs(d.D + (int64_t)__ldg(In + a) * d.ldD + __ldg(Jn + b));
    d.Dc[nb][(int64_t)a * d.ldDc + b] = v;
  }
}

// The m x R projection and reconstruction matrices of one segment (Y | X T^{-1}
// and X T^T: outputs of the core SVD, which may still be running: wait for it).
template <int R, bool COL>
__device__ __forceinline__ void pass_stage_proj(const IterDesc& d, const PassLayout& L, int k) {
  constexpr int RX = (R + 3) & ~3;
  pdl_wait();
  trace_start(d.trace, kTraceSlots * k + 3);  // the span after the wait for the SVD
  const int m = COL ? d.nJ : d.nI;
  const float* projG = COL ? d.Vs : d.W;
  for (int q = threadIdx.x; q < m * RX; q += blockDim.x) {
    const int a = q / RX, t = q - a * RX;
    const bool in = t < R;
    L.proj[q] = in ? projG[a * R + t] : 0.f;
    if (COL) L.recon[q] = in ? d.V[a * R + t] : 0.f;
  }
  __syncthreads();
}

// Tile work layout: lane l of warp h owns the column pair c0 = 2 (l & 15),
// c0 + 1, and the rows a0(h) + (l >> 4), +2, +4, ... of the warp's row share,
// so that each broadcast read of a row of the small matrices serves two
// entries and the r-wide products run as packed FP32 pairs (ffma2).

// The pair's columns of the current iterate's other factor, B_k(:,j) (row
// panel) or A_k(i,:)^T (column panel), from the tile's staged copy (zero past
// the panel's last column).
template <int R, bool COL>
__device__ __forceinline__ void pass_pair_vec(const float* lv, int c0, float2 (&vec)[R]) {
#pragma unroll
  for (int t = 0; t < R; ++t)
    vec[t] = COL ? make_float2(lv[c0 * R + t], lv[(c0 + 1) * R + t])
                 : *reinterpret_cast<const float2*>(lv + t * kPanelCols + c0);
}

// Row a of the small matrix M (RX floats a row) as R values.
template <int R>
__device__ __forceinline__ void pass_row(const float* M, int a, float (&v)[R]) {
  constexpr int RX = (R + 3) & ~3;
#pragma unroll
  for (int t4 = 0; t4 < RX / 4; ++t4) {
    const float4 q = *reinterpret_cast<const float4*>(M + (size_t)a * RX + 4 * t4);
    const float q4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * t4 + e < R) v[4 * t4 + e] = q4[e];
  }
}

// Row a of a tile, the pair's columns: the panel entries d, L_k there (the
// same FMA chain as the core, element for element), and D - S = D -
// T_zeta(D - L_k) written in place (BF16 panels: to the FP32 work buffer).
// Adds d^2 to den.  Columns past the panel's last are zero in the tile and in
// the staged factor, so they give zero.
template <int R, bool COL, bool BF>
__device__ __forceinline__ float2 pass_entry2(const IterDesc& d, const PassLayout& L, float* tileS,
                                              const uint16_t* tileH, int a, int c0, int64_t j0,
                                              const float2 (&vec)[R], float zeta, float2& den) {
  float sr[R];
  pass_row<R>(L.side, a, sr);
  const float2 l = lowrank_entry2<R>(sr, vec);
  float2* cell = reinterpret_cast<float2*>(tileS + (size_t)a * kPanelCols + c0);
  float2 dv;
  if (BF) {
    const int64_t ncolsTotal = COL ? d.n1 : d.n2;
    const uint32_t hv = *reinterpret_cast<const uint32_t*>(tileH + (size_t)a * kPanelCols + c0);
    auto fp32 = [&](int c) {
      const int64_t j = j0 + c;
      if (j >= ncolsTotal) return 0.f;
      return COL ? d.D[j * d.ldD + d.J_all[a]] : d.D[(int64_t)d.I_all[a] * d.ldD + j];
    };
    dv.x = bf16_entry((uint16_t)(hv & 0xffffu), l.x, zeta, [&]() { return fp32(c0); });
    dv.y = bf16_entry((uint16_t)(hv >> 16), l.y, zeta, [&]() { return fp32(c0 + 1); });
  } else {
    dv = *cell;
  }
  const float2 v = make_float2(panel_value(dv.x, l.x, zeta), panel_value(dv.y, l.y, zeta));
  *cell = v;
  den = ffma2(dv, dv, den);
  return v;
}

// One tile, first half: the thresholded values D - S in place and this
// thread's share of ||D||^2.  Needs only L_k, not the core SVD's outputs, so
// it runs while the SVD does.
template <int R, bool COL, bool BF, int NW>
__device__ __forceinline__ float pass_tile_threshold(const IterDesc& d, int k, float zeta, int lt,
                                                     const PassLayout& L, unsigned char* tileP, const float* lv) {
  float* tileS = BF ? L.vbuf : reinterpret_cast<float*>(tileP);
  const uint16_t* tileH = reinterpret_cast<const uint16_t*>(tileP);
  const int m = COL ? d.nJ : d.nI;
  const int lane = threadIdx.x & 31, h = threadIdx.x >> 5;
  const int c0 = 2 * (lane & 15), hr = lane >> 4;
  const int64_t j0 = (int64_t)lt * kPanelCols;
  float2 vec[R];
  pass_pair_vec<R, COL>(lv, c0, vec);
  const int a0 = h * m / NW, a1 = (h + 1) * m / NW;
  float2 den = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int a = a0 + hr; a < a1; a += 2) pass_entry2<R, COL, BF>(d, L, tileS, tileH, a, c0, j0, vec, zeta, den);
  return den.x + den.y;
}

// One tile, second half: the projections (they need the core SVD's outputs,
// staged on the segment's first tile), the next factor rows and the explicit
// residuals; this share's num/den go to wsum.  FUSE: the tile was not
// thresholded ahead of time; the threshold runs in the projection sweep and
// its ||D||^2 share is added to den.
template <int R, bool COL, bool BF, bool FUSE, int NW>
__device__ __forceinline__ void pass_tile_project(const IterDesc& d, int k, int lt, const PassLayout& L,
                                                  unsigned char* tileP, float den_in, bool stage_proj, float zeta,
                                                  const float* lv, const unsigned* lp) {
  float* tileS = BF ? L.vbuf : reinterpret_cast<float*>(tileP);
  const uint16_t* tileH = reinterpret_cast<const uint16_t*>(tileP);
  constexpr int RX = (R + 3) & ~3;
  const int m = COL ? d.nJ : d.nI;
  const int64_t ncolsTotal = COL ? d.n1 : d.n2;
  const int nxt = (k & 1) ^ 1;
  const int lane = threadIdx.x & 31, h = threadIdx.x >> 5;
  const int c0 = 2 * (lane & 15), hr = lane >> 4;
  const int64_t j0 = (int64_t)lt * kPanelCols;
  const float* proj = L.proj;
  const float* recon = COL ? L.recon : L.proj;
  const int a0 = h * m / NW, a1 = (h + 1) * m / NW;
  float2 vec[R];
  if (FUSE) pass_pair_vec<R, COL>(lv, c0, vec);
  if (COL) {
    if (stage_proj) pass_stage_proj<R, true>(d, L, k);
  } else {
    if (stage_proj) pass_stage_proj<R, false>(d, L, k);
  }
  float2 den2 = make_float2(0.f, 0.f);
  float2 acc[R];
#pragma unroll
  for (int t = 0; t < R; ++t) acc[t] = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int a = a0 + hr; a < a1; a += 2) {
    const float2 v = FUSE ? pass_entry2<R, COL, BF>(d, L, tileS, tileH, a, c0, j0, vec, zeta, den2)
                          : *reinterpret_cast<const float2*>(tileS + (size_t)a * kPanelCols + c0);
    float pr[R];
    pass_row<R>(proj, a, pr);
#pragma unroll
    for (int t = 0; t < R; ++t) acc[t] = ffma2(make_float2(pr[t], pr[t]), v, acc[t]);
  }
  // the two half-warps' rows, then this warp's share of every column
#pragma unroll
  for (int t = 0; t < R; ++t) {
    acc[t].x += __shfl_xor_sync(0xffffffffu, acc[t].x, 16);
    acc[t].y += __shfl_xor_sync(0xffffffffu, acc[t].y, 16);
  }
  if (hr == 0) {
#pragma unroll
    for (int t = 0; t < R; ++t) *reinterpret_cast<float2*>(L.part + ((size_t)h * RX + t) * kPanelCols + c0) = acc[t];
  }
  __syncthreads();
  // projections of every column: the NW share sums in a fixed order
  for (int q = threadIdx.x; q < R * kPanelCols; q += blockDim.x) {
    const int t = q / kPanelCols, cc = q - t * kPanelCols;
    float s0 = 0.f, s1 = 0.f;  // even and odd shares, then their sum (a fixed order)
#pragma unroll
    for (int hh = 0; hh < NW; hh += 2) {
      s0 += L.part[((size_t)hh * RX + t) * kPanelCols + cc];
      s1 += L.part[((size_t)(hh + 1) * RX + t) * kPanelCols + cc];
    }
    L.outS[(size_t)t * kPanelCols + cc] = s0 + s1;
  }
  __syncthreads();
  float2 out[R];
#pragma unroll
  for (int t = 0; t < R; ++t) out[t] = *reinterpret_cast<const float2*>(L.outS + (size_t)t * kPanelCols + c0);
  float2 num2 = make_float2(0.f, 0.f);
#pragma unroll 2
  for (int a = a0 + hr; a < a1; a += 2) {
    const float2 v = *reinterpret_cast<const float2*>(tileS + (size_t)a * kPanelCols + c0);
    float rr[R];
    pass_row<R>(recon, a, rr);
    float2 w = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < R; ++t) w = ffma2(make_float2(rr[t], rr[t]), out[t], w);
    const float2 e = make_float2(v.x - w.x, v.y - w.y);
    num2 = ffma2(e, e, num2);
  }
  if (h == 0 && hr == 0) {
    // the next iteration's index map entries of the pair's rows (columns)
    const int dnext = d.resample ? k + 1 : 0;
    const unsigned tag_next = (unsigned)(dnext + 1);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int64_t j = j0 + c0 + u;
      if (j >= ncolsTotal) continue;
      float o[R];
#pragma unroll
      for (int t = 0; t < R; ++t) o[t] = u ? out[t].y : out[t].x;
      if (COL) {
        float* An = d.A[nxt];
#pragma unroll
        for (int t = 0; t < R; ++t) An[j * R + t] = o[t];
      } else {
        float* Bn = d.B[nxt];
#pragma unroll
        for (int t = 0; t < R; ++t) Bn[(int64_t)t * d.n2 + j] = o[t];
      }
      // rows (columns) in the next iteration's index set also go to its
      // compact side matrix, at their position in the set
      const unsigned pos_next = lp[c0 + u];
      if (index_tag_is(pos_next, tag_next)) {
        float* side = COL ? d.AI[nxt] : d.BJt[nxt];
        const int a = index_tag_pos(pos_next);
#pragma unroll
        for (int t = 0; t < R; ++t) side[(size_t)a * R + t] = o[t];
      }
    }
  }
  // this share's sums; the tile's slot gets them in share order after the
  // block's end-of-tile barrier (pass_tile_sums)
  const float sn = warp_sum(num2.x + num2.y), sd = warp_sum(den_in + (den2.x + den2.y));
  if (lane == 0) {
    L.wsum[2 * h + 0] = sn;
    L.wsum[2 * h + 1] = sd;
  }
}

// After the end-of-tile barrier: the tile's num/den in its slot (share order).
template <int NW>
__device__ __forceinline__ void pass_tile_sums(const IterDesc& d, int gtile, const PassLayout& L) {
  if (threadIdx.x == 0) {
    float sn = 0.f, sd = 0.f;
#pragma unroll
    for (int h = 0; h < NW; ++h) {
      sn += L.wsum[2 * h + 0];
      sd += L.wsum[2 * h + 1];
    }
    d.partials[(size_t)gtile * 2 + 0] = sn;
    d.partials[(size_t)gtile * 2 + 1] = sd;
  }
}

// The block that completed an instance's last tile: e_{k+1} from the slots in
// a fixed order, then k, zeta and the loop condition.  Every slot was written
// before its block's fenced counter increment, which this block has seen:
// the slots are read from L2 with no further fence.  The kernel's completion
// orders the state writes before the next kernel and the graph's condition.
template <int NW>
__device__ void pass_finalize(const IterDesc& d, int k) {
  State* st = d.st;
  __shared__ float fin[NW][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nr = d.nRowTiles, nt = d.nRowTiles + d.nColTiles;
  const float2* slots = reinterpret_cast<const float2*>(d.partials);
  // thread q adds tiles q, q + 256, ... (row panel to a0, a1, column panel to
  // a2, a3); the loads of a group of four are all in flight together
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
  for (int b = threadIdx.x; b < nt; b += 4 * 32 * NW) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int bb = b + u * 32 * NW;
      v[u] = bb < nt ? __ldcg(slots + bb) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int bb = b + u * 32 * NW;
      if (bb < nr) {
        a0 += v[u].x;
        a1 += v[u].y;
      } else {
        a2 += v[u].x;
        a3 += v[u].y;
      }
    }
  }
  a0 = warp_sum(a0);
  a1 = warp_sum(a1);
  a2 = warp_sum(a2);
  a3 = warp_sum(a3);
  if (lane == 0) {
    fin[warp][0] = a0;
    fin[warp][1] = a1;
    fin[warp][2] = a2;
    fin[warp][3] = a3;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float f[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int w = 0; w < NW; ++w)
#pragma unroll
      for (int q = 0; q < 4; ++q) f[q] += fin[w][q];
    // e = (||row residual|| + ||column residual||) / (||D(I,:)|| + ||D(:,J)||)
    const float num = sqrtf(f[0]) + sqrtf(f[2]);
    const float den = sqrtf(f[1]) + sqrtf(f[3]);
    const double e = den > 0.f ? (double)(num / den) : 0.0;
    d.errs[k] = e;
    st->e = e;
    st->k = k + 1;
    st->zeta_last = st->zeta;
    st->zeta = st->zeta * d.gamma;
    st->counter = 0u;
    const int done = (e <= d.tol) || (k + 1 >= d.max_iter) || (st->status != 0);
    st->done = done;
    if (d.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)d.cond, done ? 0u : 1u);
  }
  __syncthreads();
}

template <int R, bool BATCH, bool BF, int NW>
__device__ __forceinline__ void pass_persistent(const IterDesc& d1, const IterDesc* __restrict__ ds,
                                                const int* __restrict__ tile_base, int count, int total,
                                                int mmax, int nbuf, unsigned char* smem) {
  constexpr int RX = (R + 3) & ~3;
  const PassLayout L = pass_layout(smem, mmax, RX, nbuf, BF, NW);
  if (!BATCH && (d1.st->done || d1.st->status)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      d1.st->done = 1;
      if (d1.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)d1.cond, 0u);
    }
    return;
  }
  // the iteration, read before any block can finalize it (kernel-span trace)
  const int k_trace = BATCH ? 0 : d1.st->k;
  if (!BATCH) trace_start(d1.trace, kTraceSlots * k_trace + 2);
  // contiguous runs, the longer ones on the lowest block indices (the blocks
  // launched last, which may start only once the SVD has left its SMs, get
  // the shorter runs)
  const int q = total / (int)gridDim.x, rem = total - q * (int)gridDim.x;
  const int bx = (int)blockIdx.x;
  const int t0 = bx * q + (bx < rem ? bx : rem);
  const int t1 = t0 + q + (bx < rem ? 1 : 0);
  if (t0 >= t1) return;
  // tile -> (instance, side, local tile); instances are visited in order
  int inst = 0;
  if (BATCH) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_base[mid] <= t0)
        lo = mid;
      else
        hi = mid - 1;
    }
    inst = lo;
  }
  // An instance's state (k, done, status) is fixed while this kernel runs:
  // only the block that completes its last tile advances it, after every
  // block has located all of its tiles.  It is read once per instance met.
  int st_inst = -1, st_active = 0, st_k = 0;
  float st_zeta = 0.f;
  auto locate = [&](int t, int& in) -> TileRef {
    if (BATCH)
      while (tile_base[in + 1] <= t) ++in;
    const IterDesc& d = BATCH ? ds[in] : d1;
    TileRef ref;
    ref.inst = in;
    const int lt = t - (BATCH ? tile_base[in] : 0);
    ref.col = lt >= d.nRowTiles;
    ref.lt = ref.col ? lt - d.nRowTiles : lt;
    if (in != st_inst) {
      st_inst = in;
      st_active = !(d.st->done || d.st->status);
      st_k = d.st->k;
      st_zeta = (float)d.st->zeta;
    }
    ref.active = st_active;
    ref.k = st_k;
    return ref;
  };
  // IRCUR-R, single instance: the index sets of this iteration in shared
  // memory, read by every tile's gathers (null: gathers read them from global)
  const int* smI = nullptr;
  const int* smJ = nullptr;
  if (!BATCH && d1.resample) {
    const int kk = locate(t0, inst).k;
    for (int q = threadIdx.x; q < d1.nI; q += blockDim.x) L.idx[q] = d1.I_all[(int64_t)kk * d1.nI + q];
    for (int q = threadIdx.x; q < d1.nJ; q += blockDim.x) L.idx[d1.nI + q] = d1.J_all[(int64_t)kk * d1.nJ + q];
    __syncthreads();
    smI = L.idx;
    smJ = L.idx + d1.nI;
  }
  // a tile and its lane data into staging buffer bi
  auto stage = [&](const TileRef& ref, int bi) {
    const IterDesc& d = BATCH ? ds[ref.inst] : d1;
    unsigned char* buf = L.tiles + (size_t)bi * L.tile_bytes;
    float* lv = L.lvec + (size_t)bi * kPanelCols * RX;
    unsigned* lp = L.lpos + (size_t)bi * kPanelCols;
    if (ref.col) {
      pass_stage_tile<true, BF>(d, ref.k, ref.lt, buf, smJ);
      pass_stage_lane<R, true>(d, ref.k, ref.lt, lv, lp);
    } else {
      pass_stage_tile<false, BF>(d, ref.k, ref.lt, buf, smI);
      pass_stage_lane<R, false>(d, ref.k, ref.lt, lv, lp);
    }
  };
  __shared__ int is_last;
  // IRCUR-R: this block's share of the next iteration's D(I,J), while the core
  // SVD runs (row tiles only)
  {
    int gin = inst;
    for (int t = t0; t < t1; ++t) {
      const TileRef ref = locate(t, gin);
      if (ref.active && !ref.col) pass_gather_next_core(BATCH ? ds[ref.inst] : d1, ref.k, ref.lt);
    }
  }
  int pin = inst;  // instance cursor of the prefetch
  TileRef cur = locate(t0, inst);
  if (cur.active) stage(cur, 0);
  cp_async_commit();
  int seg_inst = -1, seg_col = -1, seg_k = 0, run = 0;
  bool proj_staged = false;
  float zeta = 0.f;
  int early = -1;      // tile thresholded ahead of time (its den in den_early)
  float den_early = 0.f;
  for (int t = t0; t < t1; ++t) {
    if (t > t0) cur = locate(t, inst);
    const IterDesc& d = BATCH ? ds[cur.inst] : d1;
    const bool new_seg = cur.inst != seg_inst || cur.col != seg_col;
    if (new_seg && run > 0) {
      // close the previous run: count its tiles; the last one finalizes
      const IterDesc& dp = BATCH ? ds[seg_inst] : d1;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0)
        is_last = (atomicAdd(&dp.st->counter, (unsigned)run) + (unsigned)run ==
                   (unsigned)(dp.nRowTiles + dp.nColTiles));
      __syncthreads();
      if (is_last) pass_finalize<NW>(dp, seg_k);
      run = 0;
    }
    const int b = (t - t0) % nbuf;
    if (nbuf == 1 && t > t0 && cur.active) {
      stage(cur, 0);
      cp_async_commit();
    }
    bool pre = false;
    TileRef nx;
    nx.active = 0;
    if (nbuf == 2 && t + 1 < t1) {
      int in2 = pin < inst ? inst : pin;
      nx = locate(t + 1, in2);
      pin = in2;
      if (nx.active) {
        stage(nx, b ^ 1);
        pre = true;
      }
      cp_async_commit();
    }
    if (!cur.active) {
      seg_inst = cur.inst;
      seg_col = cur.col;
      continue;  // an instance that stopped: nothing to do
    }
    if (new_seg) {
      seg_inst = cur.inst;
      seg_col = cur.col;
      seg_k = cur.k;
      zeta = st_inst == cur.inst ? st_zeta : (float)d.st->zeta;
      if (cur.col)
        pass_stage_side<R, true>(d, L, seg_k);
      else
        pass_stage_side<R, false>(d, L, seg_k);
      proj_staged = false;
    }
    if (pre)
      cp_async_wait_group<1>();
    else
      cp_async_wait_group<0>();
    __syncthreads();
    unsigned char* tb = L.tiles + (size_t)b * L.tile_bytes;
    const float* lvb = L.lvec + (size_t)b * kPanelCols * RX;
    const unsigned* lpb = L.lpos + (size_t)b * kPanelCols;
    // a tile met after the segment's wait for the SVD (and not thresholded
    // ahead of time) is thresholded inside its projection sweep
    const bool fuse = proj_staged && early != t;
    float den = 0.f;
    if (early == t) {
      den = den_early;
    } else if (!fuse) {
      den = cur.col ? pass_tile_threshold<R, true, BF, NW>(d, seg_k, zeta, cur.lt, L, tb, lvb)
                    : pass_tile_threshold<R, false, BF, NW>(d, seg_k, zeta, cur.lt, L, tb, lvb);
    }
    // before the segment's first wait for the SVD: threshold the prefetched
    // next tile of the same segment as well (FP32 panels: in its own buffer)
    if (!BF && !proj_staged && pre && nx.inst == cur.inst && nx.col == cur.col) {
      cp_async_wait_group<0>();
      __syncthreads();
      unsigned char* tn = L.tiles + (size_t)(b ^ 1) * L.tile_bytes;
      const float* lvn = L.lvec + (size_t)(b ^ 1) * kPanelCols * RX;
      den_early = cur.col ? pass_tile_threshold<R, true, BF, NW>(d, seg_k, zeta, nx.lt, L, tn, lvn)
                          : pass_tile_threshold<R, false, BF, NW>(d, seg_k, zeta, nx.lt, L, tn, lvn);
      early = t + 1;
    }
    if (fuse) {
      if (cur.col)
        pass_tile_project<R, true, BF, true, NW>(d, seg_k, cur.lt, L, tb, den, false, zeta, lvb, lpb);
      else
        pass_tile_project<R, false, BF, true, NW>(d, seg_k, cur.lt, L, tb, den, false, zeta, lvb, lpb);
    } else {
      if (cur.col)
        pass_tile_project<R, true, BF, false, NW>(d, seg_k, cur.lt, L, tb, den, !proj_staged, zeta, lvb, lpb);
      else
        pass_tile_project<R, false, BF, false, NW>(d, seg_k, cur.lt, L, tb, den, !proj_staged, zeta, lvb, lpb);
    }
    proj_staged = true;
    __syncthreads();
    pass_tile_sums<NW>(d, t - (BATCH ? tile_base[cur.inst] : 0), L);
    ++run;
  }
  if (run > 0) {
    const IterDesc& dp = BATCH ? ds[seg_inst] : d1;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0)
      is_last = (atomicAdd(&dp.st->counter, (unsigned)run) + (unsigned)run == (unsigned)(dp.nRowTiles + dp.nColTiles));
    __syncthreads();
    if (is_last) pass_finalize<NW>(dp, seg_k);
  }
  cp_async_wait_group<0>();
  if (!BATCH && d1.trace) {
    __syncthreads();
    trace_stop(d1.trace, kTraceSlots * d1.max_iter, kTraceSlots * k_trace + 2);
    trace_stop(d1.trace, kTraceSlots * d1.max_iter, kTraceSlots * k_trace + 3);
  }
}

// NW warps per block; two blocks per SM up to R = 7 (64 registers a thread),
// one above (the pair layout keeps 4R FP32 values of the two columns live).
template <int R, bool BF, int NW>
__global__ void __launch_bounds__(32 * NW, R <= 7 ? 2 : 1) pass_kernel(IterDesc d, int nbuf) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int mmax = d.nI > d.nJ ? d.nI : d.nJ;
  pass_persistent<R, false, BF, NW>(d, nullptr, nullptr, 1, d.nRowTiles + d.nColTiles, mmax, nbuf, smem);
}

// Batched form: the tiles of every instance back to back (tile_base[i] is the
// first tile of instance i, tile_base[count] the total).
template <int R>
__global__ void __launch_bounds__(kPassThreads, R <= 7 ? 2 : 1) pass_batch_kernel(const IterDesc* __restrict__ ds,
                                                                  const int* __restrict__ tile_base, int count,
                                                                  int mmax, int nbuf) {
  extern __shared__ __align__(16) unsigned char smem[];
  pass_persistent<R, true, false, kPassWarps>(ds[0], ds, tile_base, count, tile_base[count], mmax, nbuf, smem);
}


// Batched loop control: the while-node continues while any instance runs.
__global__ void batch_check_kernel(const IterDesc* __restrict__ ds, int count, unsigned long long cond,
                                   int* any_active) {
  __shared__ int act;
  if (threadIdx.x == 0) act = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const State* st = ds[i].st;
    if (!st->done && !st->status) atomicOr(&act, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *any_active = act;
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, act ? 1u : 0u);
  }
}

// Shared memory of the pass kernel with nw warps per block: two tile buffers
// when they fit next to the small matrices, else one (no prefetch).
size_t pass_smem_bytes(int nI, int nJ, int Rpad, int* nbuf_out, bool bf16, bool single, int nw) {
  const int m = nI > nJ ? nI : nJ;
  const int rx = (Rpad + 3) & ~3;
  int nbuf = 2;
  size_t bytes = pass_layout_floats(m, rx, 2, bf16, nw) * 4 + 64;
  if (bytes > 227 * 1024 || single) {
    nbuf = 1;
    bytes = pass_layout_floats(m, rx, 1, bf16, nw) * 4 + 64;
  }
  if (nbuf_out) *nbuf_out = nbuf;
  return bytes;
}

// Resident blocks of a pass kernel on the current device, cached per (device,
// kernel, shared-memory size).  Solves on several host threads may ask at
// once: the cache is guarded by a mutex.
static int pass_grid(const void* fn, size_t smem, int threads) {
  struct Entry {
    int dev;
    const void* fn;
    size_t smem;
    int blocks;
  };
  static std::mutex mu;
  static Entry cache[64];
  static int ncache = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    for (int q = 0; q < ncache; ++q)
      if (cache[q].dev == dev && cache[q].fn == fn && cache[q].smem == smem) return cache[q].blocks;
  }
  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms <= 0)
    num_sms = kNumSMsHint;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int blocks = per_sm * num_sms;
  std::lock_guard<std::mutex> lock(mu);
  if (ncache < 64) cache[ncache++] = Entry{dev, fn, smem, blocks};
  return blocks;
}
cudaError_t launch_svd(const IterDesc& d, int Rpad, cudaStream_t s);

// A launch that may overlap the tail of the previous kernel in the stream
// (programmatic stream serialization; the kernel waits with pdl_wait()).
template <typename... Args>
static cudaError_t launch_pdl(void (*kernel)(Args...), int grid, int threads, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The single-instance pass kernel for R and the block's warp count, the
// shared memory it takes and its staging buffers.
template <int R>
static const void* pass_fn(const IterDesc& d, size_t* bytes, int* nbuf, int* nw) {
  const bool bf = d.bf16 != 0, single = d.passSingleBuf != 0;
  *nw = kPassWarps;
  *bytes = pass_smem_bytes(d.nI, d.nJ, R, nbuf, bf, single, *nw);
  return bf ? (const void*)pass_kernel<R, true, kPassWarps> : (const void*)pass_kernel<R, false, kPassWarps>;
}

template <int R>
static cudaError_t launch_iter_r(const IterDesc& d, cudaStream_t s) {
  {
    cudaError_t e = launch_svd(d, R, s);
    if (e != cudaSuccess) return e;
  }
  size_t bytes = 0;
  int nbuf = 1, nw = kPassWarps;
  const void* fn = pass_fn<R>(d, &bytes, &nbuf, &nw);
  const int total = d.nRowTiles + d.nColTiles;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  int grid = d.passGrid > 0 ? d.passGrid : pass_grid(fn, bytes, 32 * nw);
  if (grid > total) grid = total;
  auto kernel = reinterpret_cast<void (*)(IterDesc, int)>(const_cast<void*>(fn));
  return launch_pdl(kernel, grid, 32 * nw, bytes, s, d, nbuf);
}

template <int R>
static cudaError_t launch_batch_iter_r(const BatchLaunch& b, cudaStream_t s) {
  cudaError_t e = launch_svd_batch(b, R, s);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(pass_batch_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.pass_smem);
  if (e != cudaSuccess) return e;
  {
    int grid = b.pass_grid > 0 ? b.pass_grid : pass_grid((const void*)pass_batch_kernel<R>, b.pass_smem, kPassThreads);
    if (grid > b.total_tiles) grid = b.total_tiles;
    // a programmatic dependent of the batch's (last) core-SVD launch, as in
    // the single-instance iteration
    return launch_pdl(pass_batch_kernel<R>, grid, kPassThreads, b.pass_smem, s, b.ds, b.tile_base, b.count,
                      b.pass_mmax, b.pass_nbuf);
  }
}

// The batched pass alone, after its group's core SVD has ended (no
// programmatic overlap: its wait returns at once).
template <int R>
static cudaError_t launch_batch_pass_r(const BatchLaunch& b, cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(pass_batch_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.pass_smem);
  if (e != cudaSuccess) return e;
  int grid = b.pass_grid > 0 ? b.pass_grid : pass_grid((const void*)pass_batch_kernel<R>, b.pass_smem, kPassThreads);
  if (grid > b.total_tiles) grid = b.total_tiles;
  pass_batch_kernel<R><<<grid, kPassThreads, b.pass_smem, s>>>(b.ds, b.tile_base, b.count, b.pass_mmax, b.pass_nbuf);
  return cudaGetLastError();
}

template <int R>
static int pass_resident_r(const IterDesc& d) {
  size_t bytes = 0;
  int nbuf = 1, nw = kPassWarps;
  const void* fn = pass_fn<R>(d, &bytes, &nbuf, &nw);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return 0;
  return pass_grid(fn, bytes, 32 * nw);
}

template <int R>
static int pass_batch_resident_r(const BatchLaunch& b) {
  const void* fn = (const void*)pass_batch_kernel<R>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b.pass_smem) != cudaSuccess) return 0;
  return pass_grid(fn, b.pass_smem, kPassThreads);
}

#define IRCUR_R_DISPATCH(FN, ARG)    \
  switch (Rpad) {                    \
    case 1: return FN<1>(ARG);       \
    case 2: return FN<2>(ARG);       \
    case 3: return FN<3>(ARG);       \
    case 4: return FN<4>(ARG);       \
    case 5: return FN<5>(ARG);       \
    case 6: return FN<6>(ARG);       \
    case 7: return FN<7>(ARG);       \
    case 8: return FN<8>(ARG);       \
    case 9: return FN<9>(ARG);       \
    case 10: return FN<10>(ARG);     \
    case 12: return FN<12>(ARG);     \
    case 16: return FN<16>(ARG);     \
    case 20: return FN<20>(ARG);     \
    default: return 0;               \
  }

int pass_resident_blocks(const IterDesc& d, int Rpad) { IRCUR_R_DISPATCH(pass_resident_r, d) }
int pass_batch_resident_blocks(const BatchLaunch& b, int Rpad) { IRCUR_R_DISPATCH(pass_batch_resident_r, b) }

cudaError_t launch_batch_check(const IterDesc* ds, int count, unsigned long long cond, int* any_active,
                               cudaStream_t s) {
  batch_check_kernel<<<1, 256, 0, s>>>(ds, count, cond, any_active);
  return cudaGetLastError();
}

cudaError_t launch_batch_pass(const BatchLaunch& b, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_batch_pass_r<1>(b, s);
    case 2: return launch_batch_pass_r<2>(b, s);
    case 3: return launch_batch_pass_r<3>(b, s);
    case 4: return launch_batch_pass_r<4>(b, s);
    case 5: return launch_batch_pass_r<5>(b, s);
    case 6: return launch_batch_pass_r<6>(b, s);
    case 7: return launch_batch_pass_r<7>(b, s);
    case 8: return launch_batch_pass_r<8>(b, s);
    case 9: return launch_batch_pass_r<9>(b, s);
    case 10: return launch_batch_pass_r<10>(b, s);
    case 12: return launch_batch_pass_r<12>(b, s);
    case 16: return launch_batch_pass_r<16>(b, s);
    case 20: return launch_batch_pass_r<20>(b, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_batch_group(const BatchLaunch& b, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_batch_iter_r<1>(b, s);
    case 2: return launch_batch_iter_r<2>(b, s);
    case 3: return launch_batch_iter_r<3>(b, s);
    case 4: return launch_batch_iter_r<4>(b, s);
    case 5: return launch_batch_iter_r<5>(b, s);
    case 6: return launch_batch_iter_r<6>(b, s);
    case 7: return launch_batch_iter_r<7>(b, s);
    case 8: return launch_batch_iter_r<8>(b, s);
    case 9: return launch_batch_iter_r<9>(b, s);
    case 10: return launch_batch_iter_r<10>(b, s);
    case 12: return launch_batch_iter_r<12>(b, s);
    case 16: return launch_batch_iter_r<16>(b, s);
    case 20: return launch_batch_iter_r<20>(b, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_iteration(const IterDesc& d, int Rpad, cudaStream_t s) {
  switch (Rpad) {
    case 1: return launch_iter_r<1>(d, s);
    case 2: return launch_iter_r<2>(d, s);
    case 3: return launch_iter_r<3>(d, s);
    case 4: return launch_iter_r<4>(d, s);
    case 5: return launch_iter_r<5>(d, s);
    case 6: return launch_iter_r<6>(d, s);
    case 7: return launch_iter_r<7>(d, s);
    case 8: return launch_iter_r<8>(d, s);
    case 9: return launch_iter_r<9>(d, s);
    case 10: return launch_iter_r<10>(d, s);
    case 12: return launch_iter_r<12>(d, s);
    case 16: return launch_iter_r<16>(d, s);
    case 20: return launch_iter_r<20>(d, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ircur
