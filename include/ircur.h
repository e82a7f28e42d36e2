/*
 * ircur.h -- C ABI of libircur, a GB300 (sm_103a) implementation of IRCUR
 * (Iterated Robust CUR) for robust PCA, D = L + S, after Cai, Hamm, Huang,
 * Li, Wang, "Rapid Robust Principal Component Analysis: CUR Accelerated
 * Inexact Low Rank Estimation" (arXiv 2010.07422).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Matrices are FP32, row-major, with an explicit leading dimension (the
 *   distance in elements between the starts of consecutive rows, >= the
 *   number of columns).  "device" pointers are CUDA device (or managed)
 *   memory of the device that was current when the context was created;
 *   "host" pointers are ordinary host memory (pinned memory is faster).
 * - The caller owns every buffer it passes in; the library never frees or
 *   keeps them past the call.  The library owns only its context and the
 *   workspace the context allocates at creation.
 * - All device work is issued on the stream given to ircur_create; calls
 *   return once the work is queued, except where a call says it synchronises.
 * - Functions return an ircur_status and never abort, throw or print.
 *   IRCUR_EINVAL leaves the context unchanged; IRCUR_ECUDA means a CUDA call
 *   failed (ircur_last_error_string gives the CUDA message).
 * - Index sets are int32, sorted strictly ascending, 0-based.
 */
#ifndef IRCUR_H
#define IRCUR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IRCUR_OK = 0,
  IRCUR_EINVAL = 1,        /* bad argument, size, pointer alignment, index set, NaN/Inf in D */
  IRCUR_ENOMEM = 2,        /* workspace allocation failed */
  IRCUR_ECUDA = 3,         /* a CUDA runtime call failed */
  IRCUR_ESVD_NOCONV = 4,   /* reserved: the core SVD never returns it as an error (see flags) */
  IRCUR_ETIMEOUT = 5,      /* a bounded device wait ran out; the context stays usable */
  IRCUR_ESTATE = 6,        /* call out of order (e.g. factors before any solve) */
  IRCUR_ENOTSUP = 7        /* parameter combination not built (e.g. r > 16) */
} ircur_status;

/* ircur_result.flags bits */
#define IRCUR_FLAG_WRANK 1u        /* some core had numerical rank < r (pinv used that rank) */
#define IRCUR_FLAG_SVD_NOCONV 2u   /* the core's subspace iteration hit its step cap */
#define IRCUR_FLAG_SVD_GAP 4u      /* some core's truncated subspace stopped at the FP32 floor before its
                                      gap-scaled accuracy target: sigma_r / sigma_{r+1} too close to 1 */

/* Largest rank r this build supports. */
#define IRCUR_MAX_RANK 20

/* ircur_params.precision.
 * FP32: every panel entry, product, threshold decision and stopping-value
 *   sum in FP32 (fixed-order sums; the threshold schedule zeta_k in FP64).
 * BF16_PANELS (IRCUR-F only): the compact panels D(I,:) and D(:,J) are stored
 *   in BF16 (half their bytes); each iteration's threshold decision
 *   |D - L_k| > zeta is the FP32 one (an entry within BF16 rounding of zeta,
 *   |(|d_bf16 - l| - zeta)| <= 2^-8 |d_bf16|, is read again from the FP32 D),
 *   and every product is FP32.  The kept entries of D enter C and R rounded
 *   to BF16 (relative error <= 2^-9), so L carries an error of that order and
 *   e_k has a floor near 2^-9: pass tol >= 1e-3 or a fixed iteration count.
 *   ircur_get_cur reports C and R from the FP32 D.  Not available to
 *   batches, recording solves or ircur_solve_noalloc (ENOTSUP / EINVAL). */
#define IRCUR_PRECISION_FP32 0
#define IRCUR_PRECISION_BF16_PANELS 1

/* ircur_params.svd_form: how Phase I on the core and the rank-r truncation
 * H_r (Sec. 3.1) run on the GPU.  Both forms run the same subspace iteration
 * with the same stopping rule; their results agree to FP32 rounding, not bit
 * for bit.
 * CLUSTER: one thread-block cluster of 16 CTAs per core where the device runs
 *   clusters of 16 (a non-portable size, asked once per device), else of 8;
 *   each CTA holds a slab of the core's rows and one of its columns (the
 *   faster form for one solve).  The choice depends only on the shape and the
 *   device, so a batch instance runs the same form as a lone solve.
 * ONE_CTA: one CTA of 512 threads per core, the whole core in its shared
 *   memory, where that fits (about |I|, |J| <= 220 at r <= 8); the cluster form
 *   elsewhere.  One SM per instance instead of sixteen.
 * CLUSTER8: a cluster of 8 CTAs per core where the slabs of 8 fit (16
 *   elsewhere): for batches, where more instances then run at once. */
#define IRCUR_SVD_CLUSTER 0
#define IRCUR_SVD_ONE_CTA 1
#define IRCUR_SVD_CLUSTER8 2

/* Largest number of instances of one ircur_batch. */
#define IRCUR_MAX_BATCH 4096

typedef struct {
  int64_t n1, n2;    /* D is n1 x n2 (Alg. 1 input D) */
  int32_t r;         /* target rank r, 1 <= r <= IRCUR_MAX_RANK (Alg. 1) */
  int32_t nI, nJ;    /* |I|, |J|: r <= nI <= n1, r <= nJ <= n2 (Thm 1 needs |I|,|J| >= r);
                        0 = ceil(4 r ln n) capped at n (Sec. 3.5, c_I = 4) */
  double zeta0;      /* initial threshold zeta_0 (Alg. 1); <= 0 means max|D_ij| */
  double gamma;      /* threshold decay gamma in (0,1) (Alg. 1, Sec. 3.5) */
  double tol;        /* target precision epsilon > 0: stop once e_k <= tol (Sec. 3.3) */
  int32_t max_iter;  /* iteration cap, >= 1 (the paper loops until e_k <= tol) */
  int32_t resample;  /* 0 = IRCUR-F (fixed I,J), 1 = IRCUR-R (fresh I,J each iteration), Sec. 3.4 */
  uint64_t seed;     /* index-stream seed (used when the caller passes no index sets) */
  int32_t precision; /* IRCUR_PRECISION_*: 0 = FP32; 1 = BF16 panels (IRCUR-F only) */
  int32_t svd_form;  /* IRCUR_SVD_*: 0 = cluster (default), 1 = one CTA where the core fits, 2 = cluster of 8 */
} ircur_params;

typedef struct {
  int32_t iters;      /* iterations run, K */
  int32_t converged;  /* 1 if e_K <= tol */
  uint32_t flags;     /* IRCUR_FLAG_* */
  int32_t svd_steps;  /* products with the core (half-steps of the subspace iteration), all iterations */
  double final_err;   /* e_K, the stopping criterion of Sec. 3.3 */
  double zeta0;       /* zeta_0 actually used (max|D| when requested) */
  double zeta_next;   /* gamma^K zeta_0, the threshold ircur_reconstruct uses for S */
} ircur_result;

typedef struct ircur_ctx ircur_ctx;

/* Create a context for problems of the given shape and parameters and
 * allocate its device workspace (about 4*(n1 + n2)*(2r + |J| + |I|) bytes
 * plus max_iter*(|I|+|J|)*4 bytes of index sets).  stream: a cudaStream_t
 * (NULL = legacy default stream).  Returns EINVAL for out-of-range
 * parameters, ENOTSUP for r > IRCUR_MAX_RANK, for |I|, |J| whose core or panel
 * tiles do not fit the GPU's shared memory at the padded rank (at r = 20 a
 * core of about 440 x 440 is the largest), an unknown precision or BF16 panels
 * with resample != 0, ENOMEM if
 * the workspace cannot be allocated.  *out is NULL on failure. */
ircur_status ircur_create(const ircur_params* params, void* stream, ircur_ctx** out);

/* Release the context and its workspace (synchronises the stream first).
 * NULL is ignored. */
void ircur_destroy(ircur_ctx* ctx);

/* Run Algorithm 1 on device matrix D (n1 x n2, leading dimension ldD >= n2,
 * 4-byte aligned; 16-byte alignment of D and ldD % 4 == 0 enable the bulk-copy
 * paths).  idx_I / idx_J: optional device int32 index sets, each holding
 * (resample ? max_iter : 1) consecutive sorted sets of nI (resp. nJ)
 * indices; pass NULL for both to draw them with the library's counter-based
 * sampler (seed in params).  Both or neither must be given.  Until the loop
 * ends nothing is read back: the iterations run as one CUDA graph whose
 * while-node is driven by the device-side stopping test.  On return (the
 * call synchronises the stream) *out holds the iteration count, e_K, flags.
 * Errors: EINVAL (bad pointer/ld, unsorted or out-of-range indices, NaN or
 * Inf in D when zeta0 <= 0), ECUDA, ETIMEOUT. */
ircur_status ircur_solve(ircur_ctx* ctx, const float* D, int64_t ldD, const int32_t* idx_I,
                         const int32_t* idx_J, ircur_result* out);

/* Copy the low-rank factors of the last solve into caller buffers (device):
 * A (n1 x r, row-major, ld = r) and B (r x n2, row-major, ld = n2) with
 * L = A B = C U^+ R, A = C V_r Sigma_r^{-1}, B = W_r^T R (Thm 1 with
 * U = H_r(core) = W_r Sigma_r V_r^T).  Either pointer may be NULL.
 * ESTATE before the first solve. */
ircur_status ircur_get_factors(ircur_ctx* ctx, float* A, float* B);

/* Copy the index sets the last iteration used (device int32 buffers of nI
 * and nJ entries) and, if sigma is not NULL, the r singular values of the
 * last core (device FP32).  ESTATE before the first solve. */
ircur_status ircur_get_indices(ircur_ctx* ctx, int32_t* I, int32_t* J, float* sigma);

/* Materialise the CUR decomposition of the last iterate (Alg. 1 output
 * C_K, U_K, R_K; Thm 1: L = C U^+ R) into caller buffers (device, FP32,
 * row-major, each may be NULL): C = [D - S_K]_{:,J} (n1 x nJ, ld nJ),
 * U = H_r([D - S_K]_{I,J}) (nI x nJ, ld nJ) and R = [D - S_K]_{I,:}
 * (nI x n2, ld n2), for the index sets ircur_get_indices returns.  C and R
 * are recomputed from D (device, ldD; the matrix of the solve) with the
 * previous iterate and threshold, entry for entry as the solve formed them.
 * ESTATE before a solve. */
ircur_status ircur_get_cur(ircur_ctx* ctx, const float* D, int64_t ldD, float* C, float* U, float* R);

/* Copy the stopping-criterion history e_1..e_K of the last solve into the
 * host array errs (room for max_iter doubles); synchronises.  Returns the
 * count in *count.  ESTATE before the first solve. */
ircur_status ircur_get_errors(ircur_ctx* ctx, double* errs, int32_t* count);

/* The launch shape the context's iterations run with (no counterpart in the
 * paper; for benchmarks and reports): *svd_ctas = CTAs of one core SVD (1 for
 * the one-CTA form, else the cluster size, 8 or 16), *pass_blocks = blocks of
 * one panel-pass launch (the autotuned grid, else every block that fits the
 * GPU at once, at most one per tile), *pass_bufs = the pass's tile staging
 * buffers per block (1 or 2).  Any output pointer may be NULL.  EINVAL for a
 * NULL ctx; ECUDA if the device query fails. */
ircur_status ircur_get_launch_shape(ircur_ctx* ctx, int32_t* svd_ctas, int32_t* pass_blocks, int32_t* pass_bufs);

/* Write the dense low-rank part L = C U^+ R of the last solve into L (device,
 * n1 x n2, ldL >= n2) and, if S is not NULL, the sparse part
 * S = T_zeta(D - L) with zeta = zeta_next (the threshold the next Phase I
 * would apply; T is the hard threshold of Sec. 3.2, strict >) into S
 * (device, ldS >= n2), reading D (device, ldD).  ESTATE before a solve. */
ircur_status ircur_reconstruct(ircur_ctx* ctx, const float* D, int64_t ldD, float* L, int64_t ldL,
                               float* S, int64_t ldS);

/* Streaming extension (the paper leaves it implicit: Alg. 1 reads a column
 * only through its rows I, Sec. 3.4, and L = C U^+ R extends it to every
 * row).  New columns, for example new frames of a video (Sec. 4.2), go
 * through Alg. 1 with the last solve's C and U^+ (and its rows I) held fixed.
 * From L_0 = 0, for t < iters, with zeta_t = gamma^t zeta_0 (the solve's
 * zeta_0 and gamma):
 *   r = d_I - T_{zeta_t}(d_I - [L_t]_I),   [L_{t+1}]_I = C_{I,:} U^+ r;
 * then L = C U^+ r and S = T_{zeta_iters}(d - L) for every row.
 * Dnew: device, n1 x ncols, row-major (ldDn >= ncols), read only.  Lnew and
 * Snew (Snew may be NULL): device, n1 x ncols (ldL, ldS >= ncols), written.
 * iters <= 0 means the last solve's iteration count K.  Asynchronous on the
 * context's stream; uses a scratch of ncols * 4 * r bytes owned by the
 * context (ENOMEM if it cannot be allocated).  ESTATE before a solve; EINVAL
 * for NULL or misaligned (not 4-byte) pointers, ncols < 1 or short leading
 * dimensions; ENOTSUP for ncols > 2^21 - 32. */
ircur_status ircur_stream_columns(ircur_ctx* ctx, const float* Dnew, int64_t ldDn, int64_t ncols, int32_t iters,
                                  float* Lnew, int64_t ldL, float* Snew, int64_t ldS);

/* Whole pipeline from host memory: copy D_host (n1 x n2, ld = n2) to the
 * device, solve, reconstruct, and copy L (and S if S_host is not NULL) back
 * to host arrays of n1 x n2 (ld = n2).  Device buffers for D, L and S are
 * allocated on the first call and kept by the context.  Synchronises. */
ircur_status ircur_solve_host(ircur_ctx* ctx, const float* D_host, float* L_host, float* S_host,
                              ircur_result* out);

/* The index sampler on its own: write the sorted m-subset of [0, n) that
 * draw `draw` on axis `axis` (0 = rows, 1 = columns) of the stream `seed`
 * selects into out (device int32[m]); 1 <= m <= n < 2^31.  Element i gets
 * key splitmix64(splitmix64(splitmix64(seed) ^ (2 draw + axis)) ^ i) and
 * the m smallest keys (ties: smaller index first) are kept -- a uniform
 * m-subset, i.e. uniform sampling of Alg. 1.  stream: cudaStream_t. */
ircur_status ircur_sample_indices(uint64_t seed, int32_t draw, int32_t axis, int64_t n, int32_t m,
                                  int32_t* out, void* stream);

/* Kernel-span tracing (for profiling; off by default).  enable != 0
 * allocates a small device buffer (64 * max_iter bytes) and makes every
 * following ircur_solve record, per iteration, four spans with the device's
 * nanosecond clock, each to the last block's end of its kernel: Phase I on the
 * core (the core SVD's prologue) and the whole core SVD, from its first block's
 * start; the panel pass from its first block's start (its blocks start while
 * the core SVD runs) and from its first block's return from the wait for the
 * core SVD.  enable == 0 frees it.  The spans are measured inside the CUDA
 * graph, where host-side events cannot be placed. */
ircur_status ircur_set_trace(ircur_ctx* ctx, int32_t enable);

/* Spans of the last traced solve: span_us[4 k + {0, 1, 2, 3}] = microseconds
 * of the core's Phase I, the core SVD, the panel pass and the panel pass after
 * its wait, for iteration k (room for 4 * max_iter doubles, host); *iters = K.
 * ESTATE without tracing or solve. */
ircur_status ircur_get_trace(ircur_ctx* ctx, double* span_us, int32_t* iters);

/* Allocation-free one-shot solve: ircur_create + ircur_solve +
 * ircur_get_factors for IRCUR-F (params->resample must be 0) without any
 * device allocation.  The paper has no counterpart; this entry point exists
 * for callers that may not allocate device memory -- a process whose memory
 * pool already holds all the device memory it may use (a new cudaMalloc would
 * fail or fragment it), or a latency-bound loop that cannot afford
 * cudaMalloc's implicit synchronisation.  It runs the same kernels as
 * ircur_solve, with the workspace carved from one fixed array of device
 * memory inside the library (3.5 MB on every GPU that loads the library,
 * held until the process exits), and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 * Limits of that array: n1, n2 <= 2048, |I|, |J| <= 192, r <= 8,
 * max_iter <= 256; larger problems (and resample != 0) return IRCUR_EINVAL.
 * D: device, n1 x n2, ldD >= n2.  A (n1 x r, ld r) and B (r x n2, ld n2):
 * device outputs with L = A B.  stream: cudaStream_t.  Synchronises the
 * stream; *out as for ircur_solve.
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  The address is kept for the life of
 * the device's primary context: resetting the device (cudaDeviceReset) after
 * that first call is not supported.  All calls share the one array (its
 * contents persist between calls; each call clears what must start at
 * zero), so calls that overlap on the GPU -- from several streams or host
 * threads -- race and must not be issued. */
ircur_status ircur_solve_noalloc(const ircur_params* params, const float* D, int64_t ldD, float* A, float* B,
                                 ircur_result* out, void* stream);

/* Algorithm 2 (CUR to SVD) for the last solve's iterate L = C U^+ R:
 * L = W diag(sigma) V^T with W (n1 x r) and V (n2 x r) orthonormal and sigma
 * (r values) in descending order.  Computed from the skinny factors
 * (L = A B): one pass over A and B forming A^T A and B B^T with FP64
 * accumulation, their Cholesky factors, the SVD of the r x r product R_A R_B^T
 * (FP64 Jacobi), then W = A R_A^{-1} P and V = B^T R_B^{-1} Q -- the
 * orthonormal factors of Alg. 2's QRs are never formed.  W, V: device,
 * row-major with leading dimension r; sigma: device.  Columns beyond the
 * numerical rank have sigma = 0.  ESTATE before a solve; the first call
 * allocates a small scratch buffer (about 8 (n1 + n2) r^2 / 256 bytes). */
ircur_status ircur_get_svd(ircur_ctx* ctx, float* W, float* sigma, float* V);

/* Differentiation of unrolled IRCUR-F.
 * ircur_set_record(ctx, 1) makes the following ircur_solve calls record, for
 * every iteration k, the factors of L_k and the core's factorisation (about
 * 4 (max_iter + 1) (n1 + n2) R + 8 max_iter |I| R bytes, R = padded rank, plus
 * the adjoint's scratch of about 4 (|I| n2 + |J| n1) bytes); a recording
 * solve runs its loop from the host.  Only IRCUR-F (params.resample == 0):
 * ENOTSUP otherwise.  enable == 0 releases the buffers.  Synchronises the
 * stream. */
ircur_status ircur_set_record(ircur_ctx* ctx, int32_t enable);

/* Reverse mode of the map the last recording solve computed: Alg. 1 with the
 * fixed index sets I, J for exactly its K = iters iterations from L_0 = 0,
 * with the thresholds zeta_k = gamma^k zeta_0 held fixed, D -> (L, S) where
 * L = L_K (ircur_reconstruct's L) and S = T_{zeta_K}(D - L) (its S).
 * Given device cotangents dL, dS (n1 x n2 row-major with leading dimensions
 * lddL, lddS; either may be null = zero), writes
 *     dD = d<dL, L>/dD + d<dS, S>/dD
 * into the device array dD (n1 x n2, lddD; every entry is written).  D must
 * be the matrix of that solve (device, ldD).  The hard threshold contributes
 * its almost-everywhere derivative (its keep mask) and the rank-r truncation
 * the derivative of the truncated SVD, which exists when sigma_r > sigma_{r+1}
 * for every core (the tail coupling is solved by conjugate gradients on the
 * complements; IRCUR_ESVD_NOCONV when such a solve does not converge, i.e. the
 * gap is too small).  zeta_0 = max|D| contributes nothing (its effect is
 * through the masks only).  Returns ESTATE without a recorded solve, ENOTSUP
 * if some core had numerical rank < r (IRCUR_FLAG_WRANK).  This adjoint is
 * not in the paper.  Synchronises the stream. */
ircur_status ircur_backward(ircur_ctx* ctx, const float* D, int64_t ldD, const float* dL, int64_t lddL,
                            const float* dS, int64_t lddS, float* dD, int64_t lddD);

/* Batched solves of independent problems.  The paper solves one problem at
 * a time (Alg. 1); a batch runs Alg. 1 on `count` unrelated problems at once
 * -- each with its own shape, rank, sample sizes, thresholds, tolerance,
 * iteration cap and variant (params[i]) -- so that many problems too small to
 * fill the GPU on their own share every kernel launch (instances are grouped
 * by padded rank; each group's kernels are launched once per iteration).
 * Each instance computes exactly what ircur_create + ircur_solve with
 * params[i] (and no explicit index sets) computes, bit for bit: the same index
 * sets, iterates, stopping iteration and outputs.  An instance that meets its
 * stopping test stops while the others go on.  All instances use the stream
 * given here.
 * ircur_batch_create validates every params[i] as ircur_create does (the
 * first failure is returned) and allocates one workspace per instance.
 * count in [1, IRCUR_MAX_BATCH]. */
typedef struct ircur_batch ircur_batch;
ircur_status ircur_batch_create(const ircur_params* params, int32_t count, void* stream, ircur_batch** out);

/* Release the batch and its instances (waits for the stream). */
void ircur_batch_destroy(ircur_batch* b);

/* Solve every instance.  D: host array of `count` device pointers, D[i] the
 * n1_i x n2_i row-major data of instance i with leading dimension ldD[i]
 * (host array, ldD[i] >= n2_i).  out: host array of `count` results, each as
 * ircur_solve fills it.  Synchronises the stream.  Returns OK when every
 * instance succeeded, else the first failing instance's status (every out[i]
 * is still filled; instances that succeeded can be read).  The first solve
 * with a given set of D pointers records a CUDA graph; later solves with the
 * same pointers replay it. */
ircur_status ircur_batch_solve(ircur_batch* b, const float* const* D, const int64_t* ldD, ircur_result* out);

/* Context of instance i (owned by the batch: do not destroy it), for
 * ircur_get_factors, ircur_get_indices, ircur_get_cur, ircur_get_errors and
 * ircur_reconstruct after ircur_batch_solve.  Null for i out of range. */
ircur_ctx* ircur_batch_instance(ircur_batch* b, int32_t i);

/* Autotuning of the panel-pass launch shape (not in the paper).  The pass
 * kernel is persistent: each block walks a contiguous run of panel tiles.
 * How many blocks to launch (1, 2, ... resident blocks per SM, or one block
 * per tile) and whether each block double-buffers its tiles decide how much
 * of a tile's latency is hidden; the best choice depends on |I|, |J|, n1, n2,
 * the rank and the GPU.  ircur_autotune runs `reps` (1..16, default 3) timed
 * solves of D (device, n1 x n2, ldD) per candidate after one untimed solve,
 * and keeps the candidate with the smallest median solve time for the
 * context's later solves; *out lists what was timed.  The context's state
 * afterwards is that of the last solve run.  Synchronises the stream.
 * ircur_batch_autotune does the same for a batch (D, ldD as for
 * ircur_batch_solve). */
#define IRCUR_TUNE_MAX 8
typedef struct {
  int32_t count;                        /* candidates timed */
  int32_t chosen;                       /* index of the candidate kept */
  int32_t grid[IRCUR_TUNE_MAX];         /* pass-kernel blocks of candidate i */
  int32_t single_buffer[IRCUR_TUNE_MAX];/* 1: one tile buffer per block */
  float ms[IRCUR_TUNE_MAX];             /* median solve time of candidate i (ms) */
} ircur_tune_result;
ircur_status ircur_autotune(ircur_ctx* ctx, const float* D, int64_t ldD, int32_t reps, ircur_tune_result* out);
ircur_status ircur_batch_autotune(ircur_batch* b, const float* const* D, const int64_t* ldD, int32_t reps,
                                  ircur_tune_result* out);

/* Human-readable name of a status code (static string). */
const char* ircur_status_string(ircur_status s);

/* Message of the last CUDA error seen by this thread's calls (static
 * thread-local storage; empty if none). */
const char* ircur_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* IRCUR_H */
