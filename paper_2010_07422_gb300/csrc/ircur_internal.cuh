// Internal declarations shared by the translation units of libircur.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ircur.h"

namespace ircur {

// Number of SMs on GB300; grids of the streaming kernels are multiples of it.
constexpr int kNumSMsHint = 152;

// Upper bound of spin iterations for every device-side wait (mbarrier polls).
// A poll takes tens of nanoseconds, so this is far above any legitimate wait
// but ends a lost wait within a few seconds.
constexpr long long kSpinLimit = 1ll << 26;

// Iterations recorded per trip of the solve graph's while node: each trip
// costs a few microseconds of condition evaluation and re-launch; the kernels
// of an iteration after convergence return at once (4: 1.92 -> 1.87 ms at the
// n = 10^4, r = 5 workload).
#ifndef IRCUR_GRAPH_UNROLL
#define IRCUR_GRAPH_UNROLL 4
#endif
constexpr int kGraphUnroll = IRCUR_GRAPH_UNROLL;

// Kernel-span trace slots per iteration (ircur_set_trace): 0 Phase I on the
// core (the core SVD's prologue), 1 the core SVD, 2 the panel pass from its
// first block's start, 3 the panel pass from the first return of its wait for
// the core SVD; each to the last block's end.
constexpr int kTraceSlots = 4;

// Panel-pass tiling: a tile is kPanelCols consecutive panel columns; a block
// of kPassWarps warps computes one tile at a time, warp h owning row share h
// and lane l the column pair 2 (l & 15), 2 (l & 15) + 1 on every other row.  Each tile leaves its (num, den) partial sums in
// `partials`.
constexpr int kPanelCols = 32;
constexpr int kPassWarps = 16;
constexpr int kSvdCluster = 8;  // CTAs (SMs) of the cluster form of the core SVD
constexpr int kPassThreads = 32 * kPassWarps;
constexpr int kMaxPanelRows = 512;  // largest |I|, |J| the kernels are built for

// Device-resident solver state, written only by the kernels of one solve.
struct State {
  int k;            // iterations completed
  int done;         // 1 once e_k <= tol or k == max_iter
  int status;       // ircur_status raised on the device (0 = fine)
  unsigned flags;   // IRCUR_FLAG_*
  double zeta;      // threshold of the current iteration, zeta_0 gamma^k
  double zeta0;     // zeta_0 in use
  double zeta_last; // threshold of the last completed iteration
  double e;         // last stopping value e_k
  unsigned counter; // block-completion counter of the pass kernel
  unsigned maxabs_bits;  // max|D| as float bits (non-negative floats order like uints)
  int nonfinite;    // a NaN or Inf was seen in D
  int svd_steps;    // subspace-iteration steps, summed
  int svd_last_steps;
};

// Everything one iteration's kernels need; passed by value as a kernel
// parameter (constant bank), fixed for a captured graph.
//
// Panels.  The row panel D(I,:) is read row by row from `rowSrc`: panel row a
// is rowSrc + (rowMap ? rowMap[a] : a) * rowLd, where rowMap is the current I
// (IRCUR-R, rows of D itself) or null (IRCUR-F, the compact copy made once).
// The column panel D(:,J) is read the same way from its transpose: panel row
// b (column J_b of D) is colSrc + (colMap ? J[b] : b) * colLd, where colSrc is
// D^T (IRCUR-R, transposed once per solve) or the compact copy D(:,J)^T.
struct IterDesc {
  int64_t n1, n2;
  int r, nI, nJ, max_iter, resample;
  double gamma, tol;
  const float* D;
  int64_t ldD;
  const float* rowSrc;  // D (R) or Prow (F)
  int64_t rowLd;
  const float* colSrc;  // D^T (R) or PcolT (F)
  int64_t colLd;
  // Precision variant (IRCUR-F): the compact panels stored in BF16 (rowLd,
  // colLd are then their leading dimensions in elements); a threshold
  // decision within BF16 rounding of zeta is taken again from the FP32 D.
  int bf16;
  const uint16_t* rowSrcH;  // D(I,:) in BF16, nI x rowLd
  const uint16_t* colSrcH;  // D(:,J)^T in BF16, nJ x colLd
  float* Prow;          // F: nI x ldPr
  int64_t ldPr;
  float* PcolT;         // F: nJ x ldPc
  int64_t ldPc;
  float* DT;            // R: n2 x n1 (leading dimension ldDT)
  int64_t ldDT;
  const int* I_all;     // (resample ? max_iter : 1) x nI
  const int* J_all;     // (resample ? max_iter : 1) x nJ
  float* A[2];          // n1 x R row-major (R = padded rank of the kernels)
  float* B[2];          // R x n2 row-major
  // D(I,J) of an iteration, compact (nI x ldDc), the core SVD's Phase I
  // input.  IRCUR-F: [0] only, gathered once.  IRCUR-R:
  // iteration k reads [k & 1]; the panel pass of iteration k gathers
  // D(I_{k+1}, J_{k+1}) into [(k + 1) & 1] (the solve's prologue gathers k = 0).
  // Padding columns stay zero.
  float* Dc[2];
  int64_t ldDc;  // nJ rounded up to 4 (16-byte rows for the bulk copies)
  // Parity of the iteration this launch runs (k & 1 while the solve is still
  // iterating): known at launch (graph node u of a trip of kGraphUnroll, an
  // even count, runs k = trip kGraphUnroll + u; the host loops launch k in
  // order), so the core SVD can load the compact buffers [k & 1] before it has
  // read k.  Set by the launching code, not by the context.
  int par;
  // Index maps of the draws (k & 1 for IRCUR-R, [0] for IRCUR-F; n1 and n2
  // entries, see index_tag) and the compact side matrices of iteration k,
  // AI[k & 1] = A_k(I_k,:) (nI x R) and BJt[k & 1] = B_k(:,J_k)^T (nJ x R),
  // written through the maps by the panel pass of iteration k - 1 (zero at
  // k = 0) and read by the core SVD and the pass of iteration k.
  unsigned* posI[2];
  unsigned* posJ[2];
  float* AI[2];
  float* BJt[2];
  float* W;             // nI x R   Y: orthonormal basis of the core's dominant left subspace
  float* V;             // nJ x R   X T^T (column-pass reconstruction)
  float* Vs;            // nJ x R   X T^{-1} (column-pass projection; zero for dropped directions)
  float* sigma;         // R        |diag T| (diagnostic)
  float* Tm;            // R x R    Rayleigh-Ritz matrix T = Y^T core X of the last iteration
  float* partials;      // 2 per panel tile (row tiles, then column tiles)
  double* errs;         // max_iter
  State* st;
  int nRowTiles, nColTiles;
  int rowBulk, colBulk; // 1: panel rows are 16-byte aligned (tiles via 16-byte async copies)
  int svdMaxSteps;
  int sampleAhead;      // 1: the core-SVD launch draws the next iteration's I, J (IRCUR-R, own sampler)
  int svdNC;            // CTAs of the core SVD's cluster: 1 (one CTA), 8 or 16
  int passGrid;         // pass-kernel blocks (0: every block that fits the GPU at once), from the autotuner
  int passSingleBuf;    // 1: one tile buffer per block (no prefetch, less shared memory)
  long long spinLimit;      // first bounded wait on a bulk copy (kSpinLimit unless a fault is injected)
  unsigned long long cond;  // graph conditional handle (0 = no graph)
  unsigned long long* trace;  // optional kernel spans: slot 3k + {0 core, 1 svd, 2 pass}, 3 max_iter slots
  uint64_t seed;
};

// One iteration for a group of independent batch instances with the same
// padded rank: every kernel covers all instances of the group.
struct BatchLaunch {
  const IterDesc* ds;      // device array, one descriptor per instance
  int count;
  const int* tile_base;    // device, count + 1 prefix sums of panel tiles
  int total_tiles;
  const int* svd_list[3];  // device instance lists by core-SVD cluster size: [0] 1 CTA, [1] 8, [2] 16
  int svd_n[3];
  size_t svd_smem[3];
  int svd_roles;           // 1, or 3 when some instance draws its next index sets
  size_t pass_smem;
  int pass_mmax;           // largest |I|, |J| of the batch (shared-memory layout)
  int pass_nbuf;           // tile buffers per block (2: prefetch)
  int pass_grid;           // pass-kernel blocks (0: every block that fits the GPU at once)
  unsigned long long cond; // graph conditional handle (0 = no graph)
  int* any_active;         // device flag written by the loop-control kernel
  int par;                 // parity of the iteration launched (IterDesc::par)
};

// One reverse step k of the adjoint of unrolled IRCUR-F (k_adjoint.cu).
// The forward recorded, for every iteration k, the factors of L_k
// (A_k: n1 x R, B_k: R x n2) and the core factorisation (Y, X T^{-1}, T).
// Cotangents of L_{k+1} are carried as their projections in the forward's
// gauge, E = Gbar B_{k+1}^T (n1 x R) and F = A_{k+1}^T Gbar (R x n2).
struct AdjStep {
  int64_t n1, n2;
  int r, nI, nJ;
  const int* I;         // nI, sorted distinct
  const int* J;         // nJ
  const float* Prow;    // D(I,:), nI x ldPr
  int64_t ldPr;
  const float* PcolT;   // D(:,J)^T, nJ x ldPc
  int64_t ldPc;
  const float* Ak;      // A_k, n1 x R
  const float* Bk;      // B_k, R x n2
  const float* Y;       // nI x R
  const float* Vs;      // nJ x R, X T^{-1}
  const float* Tm;      // R x R, T(i,p) at i * R + p
  float zeta;           // zeta_k as the forward compared it (FP32)
  float* Wr;            // nI x R  exact left singular vectors W_r = Y P
  float* Vr;            // nJ x R  exact right singular vectors V_r = X Q = Vs P Sigma
  float* sig;           // R
  float* Pm;            // R x R, P(i,p) at i * R + p
  const float* E;       // n1 x R   (of L_{k+1})
  const float* F;       // R x n2
  float* Enew;          // n1 x R   (of L_k)
  float* Fnew;          // R x n2
  float* dDR;           // nI x n2, accumulated dD(I,:)
  float* dDCt;          // nJ x n1, accumulated dD(:,J)^T
  float* partR;         // nRowTiles x nI x 2R
  float* partC;         // nColTiles x nJ x 2R
  int nRowTiles, nColTiles;
  float* PhiY;          // nI x R   R_{k+1} F^T
  float* PsiY;          // nJ x R   C_{k+1}^T E
  float* e1;            // nI x R   (row-panel part of Enew(I,:))
  float* f2;            // nJ x R   (column-panel part of Fnew(:,J)^T)
  float* Ucore;         // nI x nJ scratch: the core, then its masked cotangent
  float* Xc;            // nI x R   shifted-system solutions (left complement)
  float* Yc;            // nJ x R   (right complement)
  float* G11;           // R x R
  int* status;          // set on a failed solve (IRCUR_ESVD_NOCONV)
  int cgMaxIter;
};

// Launch wrappers (return cudaGetLastError()).
// draws draw0 .. draw0 + draws - 1; with maps (two per axis, by draw parity)
// each draw also writes its index map
cudaError_t launch_sample(uint64_t seed, int draw0, int draws, int64_t n1, int64_t n2, int nI, int nJ,
                          int* I_all, int* J_all, int only_axis, cudaStream_t s, unsigned* const* mapI = nullptr,
                          unsigned* const* mapJ = nullptr);
cudaError_t launch_index_map(const int* idx, int m, unsigned* map, int draw, const State* st, cudaStream_t s);
cudaError_t launch_check_indices(const int* idx, int sets, int m, int64_t n, int* status,
                                 cudaStream_t s);
cudaError_t launch_maxabs(const float* D, int64_t n1, int64_t n2, int64_t ldD, State* st,
                          cudaStream_t s);
cudaError_t launch_transpose_maxabs(const float* D, int64_t n1, int64_t n2, int64_t ldD, float* DT,
                                    int64_t ldDT, State* st, cudaStream_t s);
cudaError_t launch_finalize_zeta(State* st, cudaStream_t s);
cudaError_t launch_setup(const IterDesc& d, double zeta0, cudaStream_t s);
cudaError_t launch_gather(const IterDesc& d, cudaStream_t s);
cudaError_t launch_iteration(const IterDesc& d, int Rpad, cudaStream_t s);
cudaError_t launch_reconstruct(const float* A, const float* B, int Rpad, int64_t n1, int64_t n2,
                               const float* D, int64_t ldD, float* L, int64_t ldL, float* S,
                               int64_t ldS, const State* st, cudaStream_t s);
cudaError_t launch_get_cur(const IterDesc& d, int Rpad, int K, const float* D, int64_t ldD, float* C, float* U,
                           float* Rm, cudaStream_t s);
// One iteration of a group of batch instances sharing a padded rank (core,
// SVD, passes), and the loop control over the whole batch.
cudaError_t launch_batch_group(const BatchLaunch& b, int Rpad, cudaStream_t s);
cudaError_t launch_batch_check(const IterDesc* ds, int count, unsigned long long cond, int* any_active,
                               cudaStream_t s);
cudaError_t launch_svd_batch(const BatchLaunch& b, int Rpad, cudaStream_t s);
// The same iteration in two phases, for batches of several rank groups: the
// core SVD alone (its look-ahead draws left to launch_sample_ahead_batch when
// svd_roles is 1), then the panel pass as a plain launch.
cudaError_t launch_batch_pass(const BatchLaunch& b, int Rpad, cudaStream_t s);
cudaError_t launch_sample_ahead_batch(const IterDesc* ds, int count, cudaStream_t s);
cudaError_t launch_stream(const float* A, const int* I, const float* Y, int m, int Rpad, int64_t n1, const float* Dn,
                          int64_t ldDn, int64_t ncols, int iters, double zeta0, double gamma, float zetaT, float* bq,
                          float* L, int64_t ldL, float* S, int64_t ldS, cudaStream_t s);
// Adjoint (k_adjoint.cu)
cudaError_t launch_adj_dense(int64_t n1, int64_t n2, const float* A, const float* B, const float* D, int64_t ldD,
                             const float* dL, int64_t lddL, const float* dS, int64_t lddS, float* dD,
                             int64_t lddD, float zetaT, float* E, float* F, int Rpad, cudaStream_t s);
cudaError_t launch_adj_step(const AdjStep& a, int Rpad, bool need_next, cudaStream_t s);
size_t adj_cg_smem_bytes(int nI, int nJ, int Rpad);
cudaError_t launch_adj_scatter(const AdjStep& a, float* dD, int64_t lddD, cudaStream_t s);
size_t pass_smem_bytes(int nI, int nJ, int Rpad, int* nbuf = nullptr, bool bf16 = false, bool single = false,
                       int nw = kPassWarps);
// Alg. 2 on the factored iterate (k_cur2svd.cu).
size_t cur_to_svd_scratch_bytes(int64_t n1, int64_t n2, int Rpad);
cudaError_t launch_cur_to_svd(const float* A, const float* B, int64_t n1, int64_t n2, int r, int Rpad, void* scratch,
                              float* W, float* sigma, float* V, cudaStream_t s);
// Core SVD (k_svd.cu): dynamic shared memory per CTA for a cluster of nc CTAs,
// whether it fits one SM, the cluster size a problem runs with on the current
// device (1 for the one-CTA form where it fits, else 16 or 8; 0 if no form
// fits), and whether some form fits at all (shape only, no CUDA call).
size_t svd_smem_bytes(int nI, int nJ, int Rpad, int nc);
bool svd_fits(int nI, int nJ, int Rpad, int nc);
int svd_cluster_size(int nI, int nJ, int Rpad, int svd_form);
bool svd_shape_ok(int nI, int nJ, int Rpad, int svd_form);
// Clusters of 16 CTAs of the largest core-SVD configuration the current device
// holds at once (k_svd_ranks_16.cu).
int svd_cluster16_capacity();
// Singular values of the last core from its T (k_svd.cu), on request.
cudaError_t launch_sigma(const float* Tm, int r, int Rpad, float* sigma, cudaStream_t s);
// D(I,J) of draw `draw` into the compact buffers [buf] (k_setup.cu).
cudaError_t launch_gather_core(const IterDesc& d, int draw, int buf, cudaStream_t s);
// Blocks of the pass kernel that are resident on the whole GPU at once.
int pass_resident_blocks(const IterDesc& d, int Rpad);
int pass_batch_resident_blocks(const BatchLaunch& b, int Rpad);
int pad_rank(int r);

}  // namespace ircur
