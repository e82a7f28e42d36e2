// Host side of libircur: the extern "C" entry points declared in ircur.h,
// workspace management, and the CUDA graph that runs Alg. 1's loop on the
// device (a conditional while-node whose body is one iteration; the pass
// kernel's last block evaluates the stopping test of Sec. 3.3 and sets the
// node's condition, so no host round trip happens inside the loop).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <memory>
#include <new>

#include "ircur.h"
#include "ircur_internal.cuh"

using namespace ircur;

namespace {

thread_local char g_last_error[256] = {0};

void set_error(const char* where, cudaError_t e) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", where, cudaGetErrorName(e),
           cudaGetErrorString(e));
}

#define IRCUR_CK(call)                       \
  do {                                       \
    cudaError_t _e = (call);                 \
    if (_e != cudaSuccess) {                 \
      set_error(#call, _e);                  \
      return IRCUR_ECUDA;                    \
    }                                        \
  } while (0)

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int default_sample_size(int r, int64_t n) {
  const double m = ceil(4.0 * r * log((double)n));
  return (int)(m < (double)n ? m : (double)n);
}

// Host-side fault injection for tests (environment variable IRCUR_FAULT):
//   alloc   -- ircur_create fails as if the workspace allocation failed,
//   svd     -- the core's subspace iteration is capped at one step,
//   timeout -- the first bounded wait of each bulk copy gets a budget of one poll.
const char* fault_mode() {
  const char* f = getenv("IRCUR_FAULT");
  return f ? f : "";
}

}  // namespace

struct ircur_ctx {
  ircur_params p;
  int Rpad;
  cudaStream_t stream;
  cudaStream_t capture_stream;
  int draws;
  // workspace
  void* ws;
  size_t ws_bytes;
  int* I_all;
  int* J_all;
  float* Prow;
  float* PcolT;
  float* DT;
  int64_t ldPr, ldPc, ldDT;
  float* A[2];
  float* B[2];
  float* Dc[2];   // D(I,J) compact (nI x ldDc); IRCUR-F uses [0] only
  int64_t ldDc;
  unsigned* posI[2];  // index maps by draw parity (IRCUR-F: [0] only)
  unsigned* posJ[2];
  float* AI[2];       // compact A_k(I_k,:), B_k(:,J_k)^T by iteration parity
  float* BJt[2];
  float* W;
  float* V;
  float* Vs;
  float* sigma;
  float* Tm;
  float* partials;
  double* errs;
  State* st;
  // graph cache
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  const float* graph_D;
  int64_t graph_ldD;
  int graph_sample_ahead;
  unsigned long long* graph_trace;
  int graph_pass_grid;
  int graph_single;
  unsigned long long* trace;  // kernel-span trace buffer (2 * kTraceSlots * max_iter), or null
  // last solve
  int solved;
  State host_state;
  // buffers of the host-memory entry point, and its copy streams / events
  float* hD;
  float* hL;
  float* hS;
  cudaStream_t hstream[4];
  cudaEvent_t hev[17];
  IterDesc desc;
  // recording forward + adjoint workspace (ircur_set_record)
  void* rec_ws;
  float* recA;   // (max_iter + 1) x n1 x R   A_k
  float* recB;   // (max_iter + 1) x R x n2   B_k
  float* recY;   // max_iter x nI x R
  float* recVs;  // max_iter x nJ x R
  float* recT;   // max_iter x R x R
  AdjStep adj;   // buffers of the reverse steps (per-step fields filled by ircur_backward)
  float* adjE[2];
  float* adjF[2];
  int recorded;  // the last solve recorded its iterations
  void* c2s_ws;  // scratch of ircur_get_svd
  float* stream_ws;       // scratch of ircur_stream_columns: one R-vector per new column
  int64_t stream_cols;    // columns it holds
};

static void reset_graph(ircur_ctx* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->exec = nullptr;
  c->graph = nullptr;
  c->graph_D = nullptr;
}

static ircur_status validate_params(const ircur_params* p, ircur_params* out) {
  if (!p) return IRCUR_EINVAL;
  ircur_params q = *p;
  if (q.n1 < 1 || q.n2 < 1 || q.n1 >= (1ll << 31) || q.n2 >= (1ll << 31)) return IRCUR_EINVAL;
  if (q.r < 1) return IRCUR_EINVAL;
  if (q.r > IRCUR_MAX_RANK) return IRCUR_ENOTSUP;
  if (q.nI == 0) q.nI = default_sample_size(q.r, q.n1);
  if (q.nJ == 0) q.nJ = default_sample_size(q.r, q.n2);
  if (q.nI < q.r || q.nJ < q.r || q.nI > q.n1 || q.nJ > q.n2) return IRCUR_EINVAL;
  if (q.nI > 512 || q.nJ > 512) return IRCUR_ENOTSUP;
  if (q.precision != IRCUR_PRECISION_FP32 && q.precision != IRCUR_PRECISION_BF16_PANELS) return IRCUR_ENOTSUP;
  if (q.precision == IRCUR_PRECISION_BF16_PANELS && q.resample != 0) return IRCUR_ENOTSUP;
  if (pass_smem_bytes(q.nI, q.nJ, pad_rank(q.r), nullptr, q.precision != 0) > 227 * 1024) return IRCUR_ENOTSUP;
  if (q.svd_form != IRCUR_SVD_CLUSTER && q.svd_form != IRCUR_SVD_ONE_CTA && q.svd_form != IRCUR_SVD_CLUSTER8)
    return IRCUR_EINVAL;
  if (!svd_shape_ok(q.nI, q.nJ, pad_rank(q.r), q.svd_form)) return IRCUR_ENOTSUP;
  if (!(q.gamma > 0.0 && q.gamma < 1.0)) return IRCUR_EINVAL;
  if (!(q.tol > 0.0)) return IRCUR_EINVAL;
  if (q.max_iter < 1) return IRCUR_EINVAL;
  if (q.resample != 0 && q.resample != 1) return IRCUR_EINVAL;
  if (!(q.zeta0 == q.zeta0)) return IRCUR_EINVAL;
  *out = q;
  return IRCUR_OK;
}

static ircur_status create_impl(const ircur_params* params, void* stream, int min_rpad, ircur_ctx** out) {
  if (!out) return IRCUR_EINVAL;
  *out = nullptr;
  ircur_params p;
  ircur_status vs = validate_params(params, &p);
  if (vs != IRCUR_OK) return vs;
  if (strcmp(fault_mode(), "alloc") == 0) return IRCUR_ENOMEM;

  ircur_ctx* c = new (std::nothrow) ircur_ctx();
  if (!c) return IRCUR_ENOMEM;
  c->p = p;
  c->Rpad = pad_rank(p.r > min_rpad ? p.r : min_rpad);
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->draws = p.resample ? p.max_iter : 1;
  const int R = c->Rpad;
  const int64_t n1 = p.n1, n2 = p.n2;
  const bool bf16 = p.precision == IRCUR_PRECISION_BF16_PANELS;
  // compact panels: FP32 rows padded to 16 bytes, or BF16 rows padded to 16 bytes
  c->ldPr = bf16 ? (n2 + 7) & ~7ll : (n2 + 3) & ~3ll;
  c->ldPc = bf16 ? (n1 + 7) & ~7ll : (n1 + 3) & ~3ll;
  const size_t pel = bf16 ? 2 : 4;
  c->ldDT = (n1 + 3) & ~3ll;

  // tile configuration of the pass kernel
  IterDesc& d = c->desc;
  memset(&d, 0, sizeof(d));
  d.svdNC = svd_cluster_size(p.nI, p.nJ, R, p.svd_form);
  if (d.svdNC == 0) {  // only a cluster of 16 fits and this device runs none
    delete c;
    return IRCUR_ENOTSUP;
  }
  d.nRowTiles = (int)((n2 + kPanelCols - 1) / kPanelCols);
  d.nColTiles = (int)((n1 + kPanelCols - 1) / kPanelCols);

  // workspace carve-up (256-byte aligned pieces)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t oI = take((size_t)c->draws * p.nI * 4);
  const size_t oJ = take((size_t)c->draws * p.nJ * 4);
  const size_t oPr = p.resample ? 0 : take((size_t)p.nI * c->ldPr * pel);
  const size_t oPc = p.resample ? 0 : take((size_t)p.nJ * c->ldPc * pel);
  const size_t oDT = p.resample ? take((size_t)n2 * c->ldDT * 4) : 0;
  const size_t oA0 = take((size_t)n1 * R * 4), oA1 = take((size_t)n1 * R * 4);
  const size_t oB0 = take((size_t)R * n2 * 4), oB1 = take((size_t)R * n2 * 4);
  c->ldDc = (p.nJ + 3) & ~3ll;
  const int ncore = p.resample ? 2 : 1;
  size_t oDc[2], oPosI[2], oPosJ[2], oAIc[2], oBJc[2];
  for (int q = 0; q < ncore; ++q) {
    oDc[q] = take((size_t)p.nI * c->ldDc * 4);
    oPosI[q] = take((size_t)n1 * 4);
    oPosJ[q] = take((size_t)n2 * 4);
  }
  for (int q = 0; q < 2; ++q) {
    oAIc[q] = take((size_t)p.nI * R * 4);
    oBJc[q] = take((size_t)p.nJ * R * 4);
  }
  const size_t oW = take((size_t)p.nI * R * 4), oV = take((size_t)p.nJ * R * 4), oVs = take((size_t)p.nJ * R * 4);
  const size_t oSig = take((size_t)R * 4);
  const size_t oTm = take((size_t)R * R * 4);
  const size_t oPart = take((size_t)(d.nRowTiles + d.nColTiles) * 2 * 4);
  const size_t oErr = take((size_t)p.max_iter * 8);
  const size_t oSt = take(sizeof(State));
  c->ws_bytes = off;
  cudaError_t e = cudaMalloc(&c->ws, c->ws_bytes);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(workspace)", e);
    cudaGetLastError();
    delete c;
    return IRCUR_ENOMEM;
  }
  e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    set_error("cudaStreamCreate", e);
    cudaFree(c->ws);
    delete c;
    return IRCUR_ECUDA;
  }
  char* base = static_cast<char*>(c->ws);
  c->I_all = reinterpret_cast<int*>(base + oI);
  c->J_all = reinterpret_cast<int*>(base + oJ);
  c->Prow = (p.resample || bf16) ? nullptr : reinterpret_cast<float*>(base + oPr);
  c->PcolT = (p.resample || bf16) ? nullptr : reinterpret_cast<float*>(base + oPc);
  if (bf16) {
    d.bf16 = 1;
    d.rowSrcH = reinterpret_cast<const uint16_t*>(base + oPr);
    d.colSrcH = reinterpret_cast<const uint16_t*>(base + oPc);
  }
  c->DT = p.resample ? reinterpret_cast<float*>(base + oDT) : nullptr;
  c->A[0] = reinterpret_cast<float*>(base + oA0);
  c->A[1] = reinterpret_cast<float*>(base + oA1);
  c->B[0] = reinterpret_cast<float*>(base + oB0);
  c->B[1] = reinterpret_cast<float*>(base + oB1);
  for (int q = 0; q < 2; ++q) {
    c->Dc[q] = reinterpret_cast<float*>(base + oDc[q < ncore ? q : 0]);
    c->posI[q] = reinterpret_cast<unsigned*>(base + oPosI[q < ncore ? q : 0]);
    c->posJ[q] = reinterpret_cast<unsigned*>(base + oPosJ[q < ncore ? q : 0]);
    c->AI[q] = reinterpret_cast<float*>(base + oAIc[q]);
    c->BJt[q] = reinterpret_cast<float*>(base + oBJc[q]);
  }
  c->W = reinterpret_cast<float*>(base + oW);
  c->V = reinterpret_cast<float*>(base + oV);
  c->Vs = reinterpret_cast<float*>(base + oVs);
  c->sigma = reinterpret_cast<float*>(base + oSig);
  c->Tm = reinterpret_cast<float*>(base + oTm);
  c->partials = reinterpret_cast<float*>(base + oPart);
  c->errs = reinterpret_cast<double*>(base + oErr);
  c->st = reinterpret_cast<State*>(base + oSt);
  e = cudaMemsetAsync(c->ws, 0, c->ws_bytes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    set_error("cudaMemset(workspace)", e);
    cudaStreamDestroy(c->capture_stream);
    cudaFree(c->ws);
    delete c;
    return IRCUR_ECUDA;
  }

  d.n1 = n1;
  d.n2 = n2;
  d.r = p.r;
  d.nI = p.nI;
  d.nJ = p.nJ;
  d.max_iter = p.max_iter;
  d.resample = p.resample;
  d.gamma = p.gamma;
  d.tol = p.tol;
  d.Prow = c->Prow;
  d.ldPr = c->ldPr;
  d.PcolT = c->PcolT;
  d.ldPc = c->ldPc;
  d.DT = c->DT;
  d.ldDT = c->ldDT;
  d.colSrc = p.resample ? c->DT : c->PcolT;
  d.colLd = p.resample ? c->ldDT : c->ldPc;
  d.colBulk = 1;
  d.I_all = c->I_all;
  d.J_all = c->J_all;
  d.A[0] = c->A[0];
  d.A[1] = c->A[1];
  d.B[0] = c->B[0];
  d.B[1] = c->B[1];
  for (int q = 0; q < 2; ++q) {
    d.Dc[q] = c->Dc[q];
    d.posI[q] = c->posI[q];
    d.posJ[q] = c->posJ[q];
    d.AI[q] = c->AI[q];
    d.BJt[q] = c->BJt[q];
  }
  d.ldDc = c->ldDc;
  d.W = c->W;
  d.V = c->V;
  d.Vs = c->Vs;
  d.sigma = c->sigma;
  d.Tm = c->Tm;
  d.partials = c->partials;
  d.errs = c->errs;
  d.st = c->st;
  d.svdMaxSteps = strcmp(fault_mode(), "svd") == 0 ? 1 : 500;
  d.spinLimit = strcmp(fault_mode(), "timeout") == 0 ? 1 : kSpinLimit;
  d.seed = p.seed;
  *out = c;
  return IRCUR_OK;
}

extern "C" ircur_status ircur_create(const ircur_params* params, void* stream, ircur_ctx** out) {
  return create_impl(params, stream, 0, out);
}

extern "C" void ircur_destroy(ircur_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  reset_graph(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->trace) cudaFree(c->trace);
  if (c->hD) cudaFree(c->hD);
  if (c->hL) cudaFree(c->hL);
  if (c->hS) cudaFree(c->hS);
  for (int q = 0; q < 4; ++q)
    if (c->hstream[q]) cudaStreamDestroy(c->hstream[q]);
  for (int q = 0; q < 17; ++q)
    if (c->hev[q]) cudaEventDestroy(c->hev[q]);
  if (c->rec_ws) cudaFree(c->rec_ws);
  if (c->c2s_ws) cudaFree(c->c2s_ws);
  if (c->stream_ws) cudaFree(c->stream_ws);
  if (c->ws) cudaFree(c->ws);
  delete c;
}

static bool use_graph() {
  const char* g = getenv("IRCUR_NO_GRAPH");
  return !(g && g[0] == '1');
}

// Build (or reuse) the graph: one conditional while-node whose body holds
// kGraphUnroll iterations (core SVD, then the panel passes, each).  The body is
// recorded by stream capture on
// the context's private stream, so any user stream (even the legacy default
// stream) can launch it.
static ircur_status build_graph(ircur_ctx* c, const IterDesc& d0) {
  reset_graph(c);
  IRCUR_CK(cudaGraphCreate(&c->graph, 0));
  cudaGraphConditionalHandle h;
  IRCUR_CK(cudaGraphConditionalHandleCreate(&h, c->graph, 1, cudaGraphCondAssignDefault));
  // cudaGraphNodeParams holds a union without a default constructor: build it
  // in zeroed raw storage.
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp->type = cudaGraphNodeTypeConditional;
  cp->conditional.handle = h;
  cp->conditional.type = cudaGraphCondTypeWhile;
  cp->conditional.size = 1;
  cudaGraphNode_t node;
  IRCUR_CK(cudaGraphAddNode(&node, c->graph, nullptr, nullptr, 0, cp));
  cudaGraph_t body = cp->conditional.phGraph_out[0];
  IterDesc d = d0;
  d.cond = (unsigned long long)h;
  IRCUR_CK(cudaStreamBeginCaptureToGraph(c->capture_stream, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
  // kGraphUnroll iterations per trip of the while node (the kernels of an
  // iteration that follows convergence return at once)
  cudaError_t le = cudaSuccess;
  static_assert(kGraphUnroll % 2 == 0, "an even unroll keeps each node's iteration parity fixed");
  for (int u = 0; u < kGraphUnroll && le == cudaSuccess; ++u) {
    IterDesc du = d;
    du.par = u & 1;
    le = launch_iteration(du, c->Rpad, c->capture_stream);
  }
  cudaGraph_t captured = nullptr;
  cudaError_t ce = cudaStreamEndCapture(c->capture_stream, &captured);
  if (le != cudaSuccess) {
    set_error("launch_iteration (capture)", le);
    reset_graph(c);
    return IRCUR_ECUDA;
  }
  if (ce != cudaSuccess) {
    set_error("cudaStreamEndCapture", ce);
    reset_graph(c);
    return IRCUR_ECUDA;
  }
  IRCUR_CK(cudaGraphInstantiate(&c->exec, c->graph, 0));
  c->graph_D = d0.D;
  c->graph_ldD = d0.ldD;
  c->graph_sample_ahead = d0.sampleAhead;
  c->graph_trace = d0.trace;
  c->graph_pass_grid = d0.passGrid;
  c->graph_single = d0.passSingleBuf;
  return IRCUR_OK;
}

static ircur_status read_state(ircur_ctx* c) {
  IRCUR_CK(cudaMemcpyAsync(&c->host_state, c->st, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
  IRCUR_CK(cudaStreamSynchronize(c->stream));
  return IRCUR_OK;
}

// Everything of a solve before the iteration loop: descriptor for this D,
// state reset, index sets, zeta_0 = max|D| (and D^T for IRCUR-R), the fixed
// panels of IRCUR-F, A_0 = B_0 = 0.  Returns the descriptor in c->desc.
// scanned: the caller has already reset the state and run the scan of D
// (max|D|, the NaN/Inf check and, for IRCUR-R, D^T) on this stream.
static ircur_status solve_prologue(ircur_ctx* c, const float* D, int64_t ldD, const int32_t* idx_I,
                                   const int32_t* idx_J, cudaStream_t s, bool scanned = false) {
  const ircur_params& p = c->p;
  if (ldD < p.n2 || (reinterpret_cast<uintptr_t>(D) & 3)) return IRCUR_EINVAL;
  if ((idx_I == nullptr) != (idx_J == nullptr)) return IRCUR_EINVAL;
  IterDesc d = c->desc;
  d.D = D;
  d.ldD = ldD;
  d.rowSrc = p.resample ? D : c->Prow;
  d.rowLd = p.resample ? ldD : c->ldPr;
  d.rowBulk = p.resample ? ((aligned16(D) && ldD % 4 == 0) ? 1 : 0) : 1;
  d.sampleAhead = (p.resample && !idx_I) ? 1 : 0;
  d.trace = c->trace;
  c->desc = d;
  c->solved = 0;
  if (c->trace) {
    const size_t half = (size_t)kTraceSlots * p.max_iter * 8;
    IRCUR_CK(cudaMemsetAsync(c->trace, 0xFF, half, s));
    IRCUR_CK(cudaMemsetAsync(reinterpret_cast<char*>(c->trace) + half, 0, half, s));
  }

  const double zeta0 = p.zeta0 > 0 ? p.zeta0 : 0.0;
  if (!scanned) IRCUR_CK(launch_setup(d, zeta0, s));
  // index maps start empty; A_0 = B_0 = 0, so A_0(I,:) and B_0(:,J) too
  const int nmap = p.resample ? 2 : 1;
  for (int q = 0; q < nmap; ++q) {
    IRCUR_CK(cudaMemsetAsync(c->posI[q], 0, (size_t)p.n1 * 4, s));
    IRCUR_CK(cudaMemsetAsync(c->posJ[q], 0, (size_t)p.n2 * 4, s));
  }
  IRCUR_CK(cudaMemsetAsync(c->AI[0], 0, (size_t)p.nI * c->Rpad * 4, s));
  IRCUR_CK(cudaMemsetAsync(c->BJt[0], 0, (size_t)p.nJ * c->Rpad * 4, s));
  // the first draws (IRCUR-R: 0 and 1, the core SVD of iteration k draws
  // k + 2) and their maps
  const int first_draws = p.resample ? (p.max_iter < 2 ? p.max_iter : 2) : 1;
  if (idx_I) {
    IRCUR_CK(cudaMemcpyAsync(c->I_all, idx_I, (size_t)c->draws * p.nI * 4, cudaMemcpyDeviceToDevice, s));
    IRCUR_CK(cudaMemcpyAsync(c->J_all, idx_J, (size_t)c->draws * p.nJ * 4, cudaMemcpyDeviceToDevice, s));
    IRCUR_CK(launch_check_indices(c->I_all, c->draws, p.nI, p.n1, &c->st->status, s));
    IRCUR_CK(launch_check_indices(c->J_all, c->draws, p.nJ, p.n2, &c->st->status, s));
    for (int q = 0; q < first_draws; ++q) {
      IRCUR_CK(launch_index_map(c->I_all + (size_t)q * p.nI, p.nI, c->posI[q & 1], q, c->st, s));
      IRCUR_CK(launch_index_map(c->J_all + (size_t)q * p.nJ, p.nJ, c->posJ[q & 1], q, c->st, s));
    }
  } else {
    IRCUR_CK(launch_sample(p.seed, 0, first_draws, p.n1, p.n2, p.nI, p.nJ, c->I_all, c->J_all, -1, s, c->posI,
                           c->posJ));
  }
  if (!scanned && p.resample) {
    // D^T for the column panels, with max|D| and the NaN/Inf scan in the same pass
    IRCUR_CK(launch_transpose_maxabs(D, p.n1, p.n2, ldD, c->DT, c->ldDT, c->st, s));
  } else if (!scanned && !(p.zeta0 > 0)) {
    IRCUR_CK(launch_maxabs(D, p.n1, p.n2, ldD, c->st, s));
  }
  if (!(p.zeta0 > 0)) IRCUR_CK(launch_finalize_zeta(c->st, s));
  if (!p.resample) IRCUR_CK(launch_gather(d, s));
  // D(I,J) of the first iteration (IRCUR-F: of every iteration) for the core SVD
  IRCUR_CK(launch_gather_core(d, 0, 0, s));
  IRCUR_CK(cudaMemsetAsync(c->A[0], 0, (size_t)p.n1 * c->Rpad * 4, s));
  IRCUR_CK(cudaMemsetAsync(c->B[0], 0, (size_t)c->Rpad * p.n2 * 4, s));
  return IRCUR_OK;
}

// The result of a solve from the device state (already read into host_state).
static ircur_status solve_epilogue(ircur_ctx* c, ircur_result* out) {
  const State& h = c->host_state;
  c->solved = 1;
  memset(out, 0, sizeof(*out));
  out->iters = h.k;
  out->converged = (h.k > 0 && h.e <= c->p.tol) ? 1 : 0;
  out->flags = h.flags;
  out->svd_steps = h.svd_steps;
  out->final_err = h.e;
  out->zeta0 = h.zeta0;
  out->zeta_next = h.zeta;
  if (h.status != 0) {
    c->solved = 0;
    return (ircur_status)h.status;
  }
  return IRCUR_OK;
}

static ircur_status solve_impl(ircur_ctx* c, const float* D, int64_t ldD, const int32_t* idx_I,
                               const int32_t* idx_J, ircur_result* out, bool scanned) {
  if (!c || !D || !out) return IRCUR_EINVAL;
  const ircur_params& p = c->p;
  ircur_status ps = solve_prologue(c, D, ldD, idx_I, idx_J, c->stream, scanned);
  if (ps != IRCUR_OK) return ps;
  const IterDesc& d = c->desc;
  cudaStream_t s = c->stream;
  c->recorded = 0;
  if (c->rec_ws) {
    // Recording forward (for ircur_backward): every iteration's factors and
    // core factorisation are copied out after it, so the loop is host-driven.
    const int R = c->Rpad;
    const size_t nA = (size_t)p.n1 * R, nB = (size_t)R * p.n2;
    IRCUR_CK(cudaMemsetAsync(c->recA, 0, nA * 4, s));
    IRCUR_CK(cudaMemsetAsync(c->recB, 0, nB * 4, s));
    for (int it = 0; it < p.max_iter; ++it) {
      IterDesc du = d;
      du.par = it & 1;
      IRCUR_CK(launch_iteration(du, R, s));
      const int nx = (it + 1) & 1;
      IRCUR_CK(cudaMemcpyAsync(c->recA + (size_t)(it + 1) * nA, c->A[nx], nA * 4, cudaMemcpyDeviceToDevice, s));
      IRCUR_CK(cudaMemcpyAsync(c->recB + (size_t)(it + 1) * nB, c->B[nx], nB * 4, cudaMemcpyDeviceToDevice, s));
      IRCUR_CK(cudaMemcpyAsync(c->recY + (size_t)it * p.nI * R, c->W, (size_t)p.nI * R * 4,
                               cudaMemcpyDeviceToDevice, s));
      IRCUR_CK(cudaMemcpyAsync(c->recVs + (size_t)it * p.nJ * R, c->Vs, (size_t)p.nJ * R * 4,
                               cudaMemcpyDeviceToDevice, s));
      IRCUR_CK(cudaMemcpyAsync(c->recT + (size_t)it * R * R, c->Tm, (size_t)R * R * 4, cudaMemcpyDeviceToDevice, s));
      if ((it & 3) == 3) {
        ircur_status rs = read_state(c);
        if (rs != IRCUR_OK) return rs;
        if (c->host_state.done) break;
      }
    }
    ircur_status rs = read_state(c);
    if (rs != IRCUR_OK) return rs;
    c->recorded = 1;
    return solve_epilogue(c, out);
  }
  if (use_graph()) {
    if (!c->exec || c->graph_D != D || c->graph_ldD != ldD || c->graph_sample_ahead != d.sampleAhead ||
        c->graph_trace != d.trace || c->graph_pass_grid != d.passGrid || c->graph_single != d.passSingleBuf) {
      ircur_status bs = build_graph(c, d);
      if (bs != IRCUR_OK) return bs;
    }
    IRCUR_CK(cudaGraphLaunch(c->exec, s));
  } else {
    // Host-driven loop (profiling and debugging: every kernel is a separate
    // launch).  The device flag is polled every few iterations.
    for (int it = 0; it < p.max_iter; ++it) {
      IterDesc du = d;
      du.par = it & 1;
      IRCUR_CK(launch_iteration(du, c->Rpad, s));
      if ((it & 3) == 3) {
        ircur_status rs = read_state(c);
        if (rs != IRCUR_OK) return rs;
        if (c->host_state.done) break;
      }
    }
  }
  ircur_status rs = read_state(c);
  if (rs != IRCUR_OK) return rs;
  return solve_epilogue(c, out);
}

extern "C" ircur_status ircur_solve(ircur_ctx* c, const float* D, int64_t ldD, const int32_t* idx_I,
                                    const int32_t* idx_J, ircur_result* out) {
  return solve_impl(c, D, ldD, idx_I, idx_J, out, false);
}

extern "C" ircur_status ircur_set_record(ircur_ctx* c, int32_t enable) {
  if (!c) return IRCUR_EINVAL;
  IRCUR_CK(cudaStreamSynchronize(c->stream));
  if (c->rec_ws) {
    cudaFree(c->rec_ws);
    c->rec_ws = nullptr;
  }
  c->recorded = 0;
  if (!enable) return IRCUR_OK;
  const ircur_params& p = c->p;
  if (p.resample || p.precision != IRCUR_PRECISION_FP32) return IRCUR_ENOTSUP;
  const int R = c->Rpad;
  const int64_t n1 = p.n1, n2 = p.n2;
  const int nI = p.nI, nJ = p.nJ, K = p.max_iter;
  if (adj_cg_smem_bytes(nI, nJ, R) > 227 * 1024) return IRCUR_ENOTSUP;
  const int nRowTiles = (int)((n2 + 31) / 32), nColTiles = (int)((n1 + 31) / 32);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t oA = take((size_t)(K + 1) * n1 * R * 4), oB = take((size_t)(K + 1) * R * n2 * 4);
  const size_t oY = take((size_t)K * nI * R * 4), oVs = take((size_t)K * nJ * R * 4), oT = take((size_t)K * R * R * 4);
  const size_t oE0 = take((size_t)n1 * R * 4), oE1 = take((size_t)n1 * R * 4);
  const size_t oF0 = take((size_t)R * n2 * 4), oF1 = take((size_t)R * n2 * 4);
  const size_t oDR = take((size_t)nI * n2 * 4), oDC = take((size_t)nJ * n1 * 4);
  const size_t oPR = take((size_t)nRowTiles * nI * 2 * R * 4), oPC = take((size_t)nColTiles * nJ * 2 * R * 4);
  const size_t oPhi = take((size_t)nI * R * 4), oPsi = take((size_t)nJ * R * 4);
  const size_t oE1v = take((size_t)nI * R * 4), oF2v = take((size_t)nJ * R * 4);
  const size_t oU = take((size_t)nI * nJ * 4);
  const size_t oXc = take((size_t)nI * R * 4), oYc = take((size_t)nJ * R * 4);
  const size_t oWr = take((size_t)nI * R * 4), oVr = take((size_t)nJ * R * 4);
  const size_t oSig = take((size_t)R * 4), oP = take((size_t)R * R * 4), oG = take((size_t)R * R * 4);
  const size_t oSt = take(16);
  cudaError_t e = cudaMalloc(&c->rec_ws, off);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(record workspace)", e);
    cudaGetLastError();
    c->rec_ws = nullptr;
    return IRCUR_ENOMEM;
  }
  e = cudaMemsetAsync(c->rec_ws, 0, off, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    set_error("cudaMemset(record workspace)", e);
    cudaFree(c->rec_ws);
    c->rec_ws = nullptr;
    return IRCUR_ECUDA;
  }
  char* b = static_cast<char*>(c->rec_ws);
  auto fp = [&](size_t o) { return reinterpret_cast<float*>(b + o); };
  c->recA = fp(oA);
  c->recB = fp(oB);
  c->recY = fp(oY);
  c->recVs = fp(oVs);
  c->recT = fp(oT);
  c->adjE[0] = fp(oE0);
  c->adjE[1] = fp(oE1);
  c->adjF[0] = fp(oF0);
  c->adjF[1] = fp(oF1);
  AdjStep& a = c->adj;
  memset(&a, 0, sizeof(a));
  a.n1 = n1;
  a.n2 = n2;
  a.r = p.r;
  a.nI = nI;
  a.nJ = nJ;
  a.I = c->I_all;
  a.J = c->J_all;
  a.Prow = c->Prow;
  a.ldPr = c->ldPr;
  a.PcolT = c->PcolT;
  a.ldPc = c->ldPc;
  a.dDR = fp(oDR);
  a.dDCt = fp(oDC);
  a.partR = fp(oPR);
  a.partC = fp(oPC);
  a.nRowTiles = nRowTiles;
  a.nColTiles = nColTiles;
  a.PhiY = fp(oPhi);
  a.PsiY = fp(oPsi);
  a.e1 = fp(oE1v);
  a.f2 = fp(oF2v);
  a.Ucore = fp(oU);
  a.Xc = fp(oXc);
  a.Yc = fp(oYc);
  a.Wr = fp(oWr);
  a.Vr = fp(oVr);
  a.sig = fp(oSig);
  a.Pm = fp(oP);
  a.G11 = fp(oG);
  a.status = reinterpret_cast<int*>(b + oSt);
  a.cgMaxIter = 200;
  return IRCUR_OK;
}

extern "C" ircur_status ircur_backward(ircur_ctx* c, const float* D, int64_t ldD, const float* dL, int64_t lddL,
                                       const float* dS, int64_t lddS, float* dD, int64_t lddD) {
  if (!c || !D || !dD) return IRCUR_EINVAL;
  if (!c->rec_ws || !c->recorded || !c->solved) return IRCUR_ESTATE;
  const ircur_params& p = c->p;
  if (ldD < p.n2 || lddD < p.n2 || (dL && lddL < p.n2) || (dS && lddS < p.n2)) return IRCUR_EINVAL;
  const State& h = c->host_state;
  const int K = h.k;
  if (K < 1) return IRCUR_ESTATE;
  if (h.flags & IRCUR_FLAG_WRANK) return IRCUR_ENOTSUP;  // a core below rank r: no derivative of H_r^+
  const int R = c->Rpad;
  cudaStream_t s = c->stream;
  AdjStep a = c->adj;
  IRCUR_CK(cudaMemsetAsync(a.dDR, 0, (size_t)p.nI * p.n2 * 4, s));
  IRCUR_CK(cudaMemsetAsync(a.dDCt, 0, (size_t)p.nJ * p.n1 * 4, s));
  IRCUR_CK(cudaMemsetAsync(a.Xc, 0, (size_t)p.nI * R * 4, s));
  IRCUR_CK(cudaMemsetAsync(a.Yc, 0, (size_t)p.nJ * R * 4, s));
  IRCUR_CK(cudaMemsetAsync(a.status, 0, 4, s));
  const size_t nA = (size_t)p.n1 * R, nB = (size_t)R * p.n2;
  // zeta_k exactly as the device formed it: zeta_0 times gamma, k times, in FP64
  double* zk = new (std::nothrow) double[K];
  if (!zk) return IRCUR_ENOMEM;
  {
    double z = h.zeta0;
    for (int k = 0; k < K; ++k) {
      zk[k] = z;
      z = z * p.gamma;
    }
  }
  int cur = 0;
  cudaError_t e = launch_adj_dense(p.n1, p.n2, c->recA + (size_t)K * nA, c->recB + (size_t)K * nB, D, ldD, dL, lddL,
                                   dS, lddS, dD, lddD, (float)h.zeta, c->adjE[cur], c->adjF[cur], R, s);
  for (int k = K - 1; k >= 0 && e == cudaSuccess; --k) {
    a.Ak = c->recA + (size_t)k * nA;
    a.Bk = c->recB + (size_t)k * nB;
    a.Y = c->recY + (size_t)k * p.nI * R;
    a.Vs = c->recVs + (size_t)k * p.nJ * R;
    a.Tm = c->recT + (size_t)k * R * R;
    a.zeta = (float)zk[k];
    a.E = c->adjE[cur];
    a.F = c->adjF[cur];
    a.Enew = c->adjE[cur ^ 1];
    a.Fnew = c->adjF[cur ^ 1];
    e = launch_adj_step(a, R, k > 0, s);
    cur ^= 1;
  }
  delete[] zk;
  if (e == cudaSuccess) e = launch_adj_scatter(a, dD, lddD, s);
  if (e != cudaSuccess) {
    set_error("ircur_backward", e);
    return IRCUR_ECUDA;
  }
  int status = 0;
  IRCUR_CK(cudaMemcpyAsync(&status, a.status, 4, cudaMemcpyDeviceToHost, s));
  IRCUR_CK(cudaStreamSynchronize(s));
  return status ? (ircur_status)status : IRCUR_OK;
}

extern "C" ircur_status ircur_get_factors(ircur_ctx* c, float* A, float* B) {
  if (!c) return IRCUR_EINVAL;
  if (!c->solved) return IRCUR_ESTATE;
  const int K = c->host_state.k;
  const int R = c->Rpad, r = c->p.r;
  if (A)
    IRCUR_CK(cudaMemcpy2DAsync(A, (size_t)r * 4, c->A[K & 1], (size_t)R * 4, (size_t)r * 4, (size_t)c->p.n1,
                               cudaMemcpyDeviceToDevice, c->stream));
  if (B)
    IRCUR_CK(cudaMemcpyAsync(B, c->B[K & 1], (size_t)r * c->p.n2 * 4, cudaMemcpyDeviceToDevice, c->stream));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_get_svd(ircur_ctx* c, float* W, float* sigma, float* V) {
  if (!c || !W || !sigma || !V) return IRCUR_EINVAL;
  if (!c->solved) return IRCUR_ESTATE;
  const ircur_params& p = c->p;
  if (!c->c2s_ws) {
    cudaError_t e = cudaMalloc(&c->c2s_ws, cur_to_svd_scratch_bytes(p.n1, p.n2, c->Rpad));
    if (e != cudaSuccess) {
      set_error("cudaMalloc(ircur_get_svd scratch)", e);
      cudaGetLastError();
      c->c2s_ws = nullptr;
      return IRCUR_ENOMEM;
    }
  }
  const int K = c->host_state.k;
  IRCUR_CK(launch_cur_to_svd(c->A[K & 1], c->B[K & 1], p.n1, p.n2, p.r, c->Rpad, c->c2s_ws, W, sigma, V, c->stream));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_get_indices(ircur_ctx* c, int32_t* I, int32_t* J, float* sigma) {
  if (!c) return IRCUR_EINVAL;
  if (!c->solved) return IRCUR_ESTATE;
  const int K = c->host_state.k;
  const int draw = c->p.resample ? (K > 0 ? K - 1 : 0) : 0;
  if (I)
    IRCUR_CK(cudaMemcpyAsync(I, c->I_all + (size_t)draw * c->p.nI, (size_t)c->p.nI * 4, cudaMemcpyDeviceToDevice,
                             c->stream));
  if (J)
    IRCUR_CK(cudaMemcpyAsync(J, c->J_all + (size_t)draw * c->p.nJ, (size_t)c->p.nJ * 4, cudaMemcpyDeviceToDevice,
                             c->stream));
  if (sigma) IRCUR_CK(launch_sigma(c->Tm, c->p.r, c->Rpad, sigma, c->stream));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_get_cur(ircur_ctx* c, const float* D, int64_t ldD, float* C, float* U, float* R) {
  if (!c || !D) return IRCUR_EINVAL;
  if (!c->solved || c->host_state.k < 1) return IRCUR_ESTATE;
  if (ldD < c->p.n2 || (reinterpret_cast<uintptr_t>(D) & 3)) return IRCUR_EINVAL;
  if (!C && !U && !R) return IRCUR_OK;
  IRCUR_CK(launch_get_cur(c->desc, c->Rpad, c->host_state.k, D, ldD, C, U, R, c->stream));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_get_errors(ircur_ctx* c, double* errs, int32_t* count) {
  if (!c || !errs || !count) return IRCUR_EINVAL;
  if (!c->solved) return IRCUR_ESTATE;
  const int K = c->host_state.k;
  if (K > 0) IRCUR_CK(cudaMemcpyAsync(errs, c->errs, (size_t)K * 8, cudaMemcpyDeviceToHost, c->stream));
  IRCUR_CK(cudaStreamSynchronize(c->stream));
  *count = K;
  return IRCUR_OK;
}

extern "C" ircur_status ircur_get_launch_shape(ircur_ctx* c, int32_t* svd_ctas, int32_t* pass_blocks,
                                               int32_t* pass_bufs) {
  if (!c) return IRCUR_EINVAL;
  const IterDesc& d = c->desc;
  if (svd_ctas) *svd_ctas = d.svdNC;
  int nbuf = 1;
  pass_smem_bytes(d.nI, d.nJ, c->Rpad, &nbuf, d.bf16 != 0, d.passSingleBuf != 0);
  if (pass_bufs) *pass_bufs = nbuf;
  if (pass_blocks) {
    int g = d.passGrid > 0 ? d.passGrid : pass_resident_blocks(d, c->Rpad);
    if (g <= 0) return IRCUR_ECUDA;
    const int total = d.nRowTiles + d.nColTiles;
    *pass_blocks = g < total ? g : total;
  }
  return IRCUR_OK;
}

extern "C" ircur_status ircur_stream_columns(ircur_ctx* c, const float* Dnew, int64_t ldDn, int64_t ncols,
                                             int32_t iters, float* Lnew, int64_t ldL, float* Snew, int64_t ldS) {
  if (!c || !Dnew || !Lnew || ncols < 1) return IRCUR_EINVAL;
  if (!c->solved || c->host_state.k < 1) return IRCUR_ESTATE;
  if (ldDn < ncols || ldL < ncols || (Snew && ldS < ncols)) return IRCUR_EINVAL;
  if ((reinterpret_cast<uintptr_t>(Dnew) & 3) || (reinterpret_cast<uintptr_t>(Lnew) & 3) ||
      (reinterpret_cast<uintptr_t>(Snew) & 3))
    return IRCUR_EINVAL;
  if (ncols > 65535ll * 32 || c->p.n1 > (1ll << 33)) return IRCUR_ENOTSUP;  // grid of the dense kernel
  const int K = c->host_state.k;
  if (iters <= 0) iters = K;
  if (c->stream_cols < ncols) {
    if (c->stream_ws) cudaFree(c->stream_ws);
    c->stream_ws = nullptr;
    c->stream_cols = 0;
    cudaError_t e = cudaMalloc(&c->stream_ws, (size_t)ncols * c->Rpad * 4);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(stream scratch)", e);
      cudaGetLastError();
      c->stream_ws = nullptr;
      return IRCUR_ENOMEM;
    }
    c->stream_cols = ncols;
  }
  const ircur_params& p = c->p;
  const int draw = p.resample ? K - 1 : 0;  // the rows I of the final iterate
  const int* I = c->desc.I_all + (int64_t)draw * p.nI;
  const double zeta0 = c->host_state.zeta0;
  double zT = zeta0;  // zeta_0 gamma^iters, the threshold of S
  for (int t = 0; t < iters; ++t) zT *= p.gamma;
  IRCUR_CK(launch_stream(c->A[K & 1], I, c->desc.W, p.nI, c->Rpad, p.n1, Dnew, ldDn, ncols, iters, zeta0, p.gamma,
                         (float)zT, c->stream_ws, Lnew, ldL, Snew, ldS, c->stream));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_reconstruct(ircur_ctx* c, const float* D, int64_t ldD, float* L, int64_t ldL,
                                          float* S, int64_t ldS) {
  if (!c || !L) return IRCUR_EINVAL;
  if (!c->solved) return IRCUR_ESTATE;
  const ircur_params& p = c->p;
  if (ldL < p.n2 || (reinterpret_cast<uintptr_t>(L) & 3)) return IRCUR_EINVAL;
  if (p.n1 > 65535ll * 16) return IRCUR_ENOTSUP;  // grid.y of the reconstruction kernel
  if (S && (!D || ldS < p.n2 || ldD < p.n2 || (reinterpret_cast<uintptr_t>(S) & 3) ||
            (reinterpret_cast<uintptr_t>(D) & 3)))
    return IRCUR_EINVAL;
  const int K = c->host_state.k;
  IRCUR_CK(launch_reconstruct(c->A[K & 1], c->B[K & 1], c->Rpad, p.n1, p.n2, D, ldD, L, ldL, S, ldS, c->st,
                              c->stream));
  return IRCUR_OK;
}

// Host-memory entry point.  The copies are pipelined over four copy streams:
// D goes up in row chunks, each scanned as soon as it has landed (max|D|, the
// NaN/Inf check and, for IRCUR-R, its columns of D^T) while the next chunks
// are still on their way; the iterations wait for all of them.  L and S are
// reconstructed chunk by chunk, each chunk's rows going back while the next
// chunk is computed.  Chunks start on multiples of 64 rows (the transpose's
// tile), so that every chunk's part of D^T starts on a 16-byte boundary.
extern "C" ircur_status ircur_solve_host(ircur_ctx* c, const float* D_host, float* L_host, float* S_host,
                                         ircur_result* out) {
  if (!c || !D_host || !L_host || !out) return IRCUR_EINVAL;
  const ircur_params& p = c->p;
  const size_t bytes = (size_t)p.n1 * p.n2 * 4;
  constexpr int kCopyStreams = 4, kChunks = 8;
  if (!c->hD) {
    cudaError_t e = cudaMalloc(&c->hD, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->hL, bytes);
    for (int q = 0; q < kCopyStreams && e == cudaSuccess; ++q)
      e = cudaStreamCreateWithFlags(&c->hstream[q], cudaStreamNonBlocking);
    for (int q = 0; q < 2 * kChunks + 1 && e == cudaSuccess; ++q)
      e = cudaEventCreateWithFlags(&c->hev[q], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      set_error("host-path buffers, streams and events", e);
      cudaGetLastError();
      return IRCUR_ENOMEM;
    }
  }
  if (S_host && !c->hS) {
    cudaError_t e = cudaMalloc(&c->hS, bytes);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(host-path S)", e);
      cudaGetLastError();
      return IRCUR_ENOMEM;
    }
  }
  const int64_t n2 = p.n2;
  const int64_t rows = ((p.n1 + kChunks - 1) / kChunks + 63) / 64 * 64;
  // the state reset comes before the first scan (the scans accumulate max|D|)
  IRCUR_CK(launch_setup(c->desc, p.zeta0 > 0 ? p.zeta0 : 0.0, c->stream));
  // D up: the copy streams start after earlier work on the context's stream
  IRCUR_CK(cudaEventRecord(c->hev[2 * kChunks], c->stream));
  for (int q = 0; q < kChunks; ++q) {
    const int64_t r0 = q * rows;
    const int64_t nr = p.n1 - r0 < rows ? p.n1 - r0 : rows;
    if (nr <= 0) break;
    cudaStream_t cs = c->hstream[q % kCopyStreams];
    IRCUR_CK(cudaStreamWaitEvent(cs, c->hev[2 * kChunks], 0));
    IRCUR_CK(cudaMemcpyAsync(c->hD + r0 * n2, D_host + r0 * n2, (size_t)nr * n2 * 4, cudaMemcpyHostToDevice, cs));
    IRCUR_CK(cudaEventRecord(c->hev[q], cs));
    IRCUR_CK(cudaStreamWaitEvent(c->stream, c->hev[q], 0));
    if (p.resample)
      IRCUR_CK(launch_transpose_maxabs(c->hD + r0 * n2, nr, n2, n2, c->DT + r0, c->ldDT, c->st, c->stream));
    else if (!(p.zeta0 > 0))
      IRCUR_CK(launch_maxabs(c->hD + r0 * n2, nr, n2, n2, c->st, c->stream));
  }
  ircur_status s = solve_impl(c, c->hD, n2, nullptr, nullptr, out, true);
  if (s != IRCUR_OK) return s;
  // L (and S) down, chunk by chunk behind the reconstruction
  const int K = c->host_state.k;
  const float* A = c->A[K & 1];
  for (int q = 0; q < kChunks; ++q) {
    const int64_t r0 = q * rows;
    const int64_t nr = p.n1 - r0 < rows ? p.n1 - r0 : rows;
    if (nr <= 0) break;
    IRCUR_CK(launch_reconstruct(A + r0 * c->Rpad, c->B[K & 1], c->Rpad, nr, n2, c->hD + r0 * n2, n2,
                                c->hL + r0 * n2, n2, S_host ? c->hS + r0 * n2 : nullptr, n2, c->st, c->stream));
    IRCUR_CK(cudaEventRecord(c->hev[kChunks + q], c->stream));
    cudaStream_t cs = c->hstream[q % kCopyStreams];
    IRCUR_CK(cudaStreamWaitEvent(cs, c->hev[kChunks + q], 0));
    IRCUR_CK(cudaMemcpyAsync(L_host + r0 * n2, c->hL + r0 * n2, (size_t)nr * n2 * 4, cudaMemcpyDeviceToHost, cs));
    if (S_host)
      IRCUR_CK(cudaMemcpyAsync(S_host + r0 * n2, c->hS + r0 * n2, (size_t)nr * n2 * 4, cudaMemcpyDeviceToHost, cs));
  }
  for (int q = 0; q < kCopyStreams; ++q) IRCUR_CK(cudaStreamSynchronize(c->hstream[q]));
  IRCUR_CK(cudaStreamSynchronize(c->stream));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_sample_indices(uint64_t seed, int32_t draw, int32_t axis, int64_t n, int32_t m,
                                             int32_t* out, void* stream) {
  if (!out || m < 1 || n < m || n >= (1ll << 31) || (axis != 0 && axis != 1) || draw < 0) return IRCUR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (axis == 0)
    IRCUR_CK(launch_sample(seed, draw, 1, n, 1, m, 1, out, nullptr, 0, s));
  else
    IRCUR_CK(launch_sample(seed, draw, 1, 1, n, 1, m, nullptr, out, 1, s));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_set_trace(ircur_ctx* c, int32_t enable) {
  if (!c) return IRCUR_EINVAL;
  if (enable && !c->trace) {
    cudaError_t e = cudaMalloc(&c->trace, (size_t)2 * kTraceSlots * c->p.max_iter * 8);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(trace)", e);
      cudaGetLastError();
      c->trace = nullptr;
      return IRCUR_ENOMEM;
    }
  } else if (!enable && c->trace) {
    IRCUR_CK(cudaStreamSynchronize(c->stream));
    cudaFree(c->trace);
    c->trace = nullptr;
  }
  return IRCUR_OK;
}

extern "C" ircur_status ircur_get_trace(ircur_ctx* c, double* span_us, int32_t* iters) {
  if (!c || !span_us || !iters) return IRCUR_EINVAL;
  if (!c->trace || !c->solved) return IRCUR_ESTATE;
  const int n = kTraceSlots * c->p.max_iter;
  unsigned long long* h = new (std::nothrow) unsigned long long[2 * (size_t)n];
  if (!h) return IRCUR_ENOMEM;
  cudaError_t e = cudaMemcpyAsync(h, c->trace, (size_t)2 * n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    delete[] h;
    set_error("ircur_get_trace", e);
    return IRCUR_ECUDA;
  }
  const int K = c->host_state.k;
  for (int q = 0; q < kTraceSlots * K; ++q)
    span_us[q] = (h[n + q] >= h[q] && h[q] != ~0ull) ? (double)(h[n + q] - h[q]) * 1e-3 : 0.0;
  *iters = K;
  delete[] h;
  return IRCUR_OK;
}

extern "C" const char* ircur_status_string(ircur_status s) {
  switch (s) {
    case IRCUR_OK: return "IRCUR_OK";
    case IRCUR_EINVAL: return "IRCUR_EINVAL: invalid argument";
    case IRCUR_ENOMEM: return "IRCUR_ENOMEM: device allocation failed";
    case IRCUR_ECUDA: return "IRCUR_ECUDA: CUDA runtime error";
    case IRCUR_ESVD_NOCONV: return "IRCUR_ESVD_NOCONV: core SVD did not converge";
    case IRCUR_ETIMEOUT: return "IRCUR_ETIMEOUT: bounded device wait expired";
    case IRCUR_ESTATE: return "IRCUR_ESTATE: call out of order";
    case IRCUR_ENOTSUP: return "IRCUR_ENOTSUP: configuration not supported by this build";
  }
  return "IRCUR_UNKNOWN";
}

extern "C" const char* ircur_last_error_string(void) { return g_last_error; }

// ---------------------------------------------------------------------------
// Batches of independent problems (each with its own shape, rank, sample
// sizes and variant) solved together.  Instances are grouped by padded rank;
// every iteration launches each group's kernels once (the core and SVD
// launches index the instance by a grid dimension, the pass launch lays the
// group's tiles end to end), and a one-block kernel ends the loop once every
// instance has met its own stopping test (instances that stopped skip their
// blocks).  Each instance keeps its own padded rank, so it computes exactly
// what a lone solve computes.

constexpr int kMaxRankGroups = 16;

struct ircur_batch {
  int count;
  int max_iter;  // the largest max_iter of the batch
  cudaStream_t stream;
  cudaStream_t capture_stream;
  cudaStream_t body_stream;
  ircur_ctx** inst;  // user order
  int* order;        // position in the descriptor array -> user index
  int* pos;          // user index -> position
  IterDesc* hdesc;   // descriptor array order
  void* dws;         // device: descriptors, tile prefix sums, SVD lists, loop flag
  IterDesc* ds;      // device descriptors (grouped order)
  int* any_active;
  State* hstates;    // pinned host copies of the states (descriptor order)
  int ngroups;
  int grpR[kMaxRankGroups];      // padded rank of group g
  int grpFirst[kMaxRankGroups];  // its first position in the descriptor array
  BatchLaunch grp[kMaxRankGroups];
  cudaStream_t gstream[kMaxRankGroups];  // one branch per group (they run concurrently)
  cudaEvent_t gev[kMaxRankGroups + 1];
  // several groups, IRCUR-R: the look-ahead draws on a branch of their own
  bool sample_branch;
  cudaStream_t sstream;
  cudaEvent_t sev;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  const float** graph_D;  // the D pointers and leading dimensions the graph was built for
  int64_t* graph_ld;
};

static void batch_reset_graph(ircur_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

extern "C" void ircur_batch_destroy(ircur_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_reset_graph(b);
  if (b->inst) {
    for (int i = 0; i < b->count; ++i) ircur_destroy(b->inst[i]);
    delete[] b->inst;
  }
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->body_stream) cudaStreamDestroy(b->body_stream);
  for (int g = 0; g < kMaxRankGroups; ++g)
    if (b->gstream[g]) cudaStreamDestroy(b->gstream[g]);
  for (int g = 0; g <= kMaxRankGroups; ++g)
    if (b->gev[g]) cudaEventDestroy(b->gev[g]);
  if (b->sstream) cudaStreamDestroy(b->sstream);
  if (b->sev) cudaEventDestroy(b->sev);
  if (b->dws) cudaFree(b->dws);
  if (b->hstates) cudaFreeHost(b->hstates);
  delete[] b->hdesc;
  delete[] b->order;
  delete[] b->pos;
  delete[] b->graph_D;
  delete[] b->graph_ld;
  delete b;
}

extern "C" ircur_status ircur_batch_create(const ircur_params* params, int32_t count, void* stream,
                                           ircur_batch** out) {
  if (!out) return IRCUR_EINVAL;
  *out = nullptr;
  if (!params || count < 1 || count > IRCUR_MAX_BATCH) return IRCUR_EINVAL;
  for (int i = 0; i < count; ++i) {
    ircur_params q;
    ircur_status vs = validate_params(&params[i], &q);
    if (vs != IRCUR_OK) return vs;
    if (q.precision != IRCUR_PRECISION_FP32) return IRCUR_ENOTSUP;
  }
  ircur_batch* b = new (std::nothrow) ircur_batch();
  if (!b) return IRCUR_ENOMEM;
  b->count = count;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->inst = new (std::nothrow) ircur_ctx*[count]();
  b->order = new (std::nothrow) int[count];
  b->pos = new (std::nothrow) int[count];
  b->hdesc = new (std::nothrow) IterDesc[count];
  b->graph_D = new (std::nothrow) const float*[count]();
  b->graph_ld = new (std::nothrow) int64_t[count]();
  if (!b->inst || !b->order || !b->pos || !b->hdesc || !b->graph_D || !b->graph_ld) {
    ircur_batch_destroy(b);
    return IRCUR_ENOMEM;
  }
  for (int i = 0; i < count; ++i) {
    ircur_status cs = create_impl(&params[i], stream, 0, &b->inst[i]);
    if (cs != IRCUR_OK) {
      ircur_batch_destroy(b);
      return cs;
    }
  }
  // descriptor order: by padded rank (stable), one group per padded rank
  {
    int n = 0;
    for (int rp = 1; rp <= IRCUR_MAX_RANK; ++rp) {
      const int first = n;
      for (int i = 0; i < count; ++i)
        if (b->inst[i]->Rpad == rp) b->order[n++] = i;
      if (n > first) {
        b->grpR[b->ngroups] = rp;
        b->grpFirst[b->ngroups] = first;
        b->grp[b->ngroups].count = n - first;
        ++b->ngroups;
      }
    }
    for (int q = 0; q < count; ++q) b->pos[b->order[q]] = q;
  }
  // device workspace: descriptors | per-group tile prefix sums | instance list | loop flag
  const size_t oDesc = 0;
  const size_t oTiles = (oDesc + (size_t)count * sizeof(IterDesc) + 255) & ~(size_t)255;
  const size_t oList = (oTiles + (size_t)(count + b->ngroups) * 4 + 255) & ~(size_t)255;
  const size_t oFlag = (oList + (size_t)count * 4 + 255) & ~(size_t)255;
  const size_t bytes = oFlag + 256;
  std::unique_ptr<int[]> tiles(new int[count + b->ngroups]);
  // per group: the instances by the cluster size of their core SVD
  std::unique_ptr<int[]> lists(new int[count]);
  cudaError_t e = cudaMalloc(&b->dws, bytes);
  if (e != cudaSuccess) {
    set_error("cudaMalloc(batch workspace)", e);
    cudaGetLastError();
    ircur_batch_destroy(b);
    return IRCUR_ENOMEM;
  }
  char* base = static_cast<char*>(b->dws);
  b->ds = reinterpret_cast<IterDesc*>(base + oDesc);
  b->any_active = reinterpret_cast<int*>(base + oFlag);
  for (int g = 0; g < b->ngroups; ++g) {
    BatchLaunch& bl = b->grp[g];
    const int first = b->grpFirst[g], n = bl.count, R = b->grpR[g];
    memset(&bl, 0, sizeof(bl));
    bl.count = n;
    bl.ds = b->ds + first;
    int* tb = tiles.get() + first + g;
    tb[0] = 0;
    int roles = 1;
    // instances by core-SVD cluster size (1, 8, 16), in group order within each
    int nf[3] = {0, 0, 0};
    auto form_of = [](int nc) { return nc == 1 ? 0 : (nc == kSvdCluster ? 1 : 2); };
    for (int q = 0; q < n; ++q) ++nf[form_of(b->inst[b->order[first + q]]->desc.svdNC)];
    int fill[3] = {0, nf[0], nf[0] + nf[1]};
    for (int q = 0; q < n; ++q) {
      const ircur_ctx* c = b->inst[b->order[first + q]];
      const ircur_params& p = c->p;
      const int f = form_of(c->desc.svdNC);
      const size_t ss = svd_smem_bytes(p.nI, p.nJ, R, c->desc.svdNC);
      if (pass_smem_bytes(p.nI, p.nJ, R) > 227 * 1024 || ss > 227 * 1024) {
        ircur_batch_destroy(b);
        return IRCUR_ENOTSUP;
      }
      if (ss > bl.svd_smem[f]) bl.svd_smem[f] = ss;
      lists[first + fill[f]++] = q;  // group-relative instance indices
      if (p.nI > bl.pass_mmax) bl.pass_mmax = p.nI;
      if (p.nJ > bl.pass_mmax) bl.pass_mmax = p.nJ;
      const int64_t t = (int64_t)tb[q] + c->desc.nRowTiles + c->desc.nColTiles;
      if (t > (1ll << 30)) {
        ircur_batch_destroy(b);
        return IRCUR_ENOTSUP;
      }
      tb[q + 1] = (int)t;
      if (p.resample) roles = 3;
      if (p.max_iter > b->max_iter) b->max_iter = p.max_iter;
    }
    bl.tile_base = reinterpret_cast<const int*>(base + oTiles) + first + g;
    bl.total_tiles = tb[n];
    bl.pass_smem = pass_smem_bytes(bl.pass_mmax, bl.pass_mmax, R, &bl.pass_nbuf);
    bl.svd_list[0] = reinterpret_cast<const int*>(base + oList) + first;
    bl.svd_list[1] = bl.svd_list[0] + nf[0];
    bl.svd_list[2] = bl.svd_list[1] + nf[1];
    for (int f = 0; f < 3; ++f) bl.svd_n[f] = nf[f];
    bl.svd_roles = roles;
    bl.cond = 0;
    bl.any_active = b->any_active;
  }
  e = cudaMallocHost(reinterpret_cast<void**>(&b->hstates), (size_t)count * sizeof(State));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->body_stream, cudaStreamNonBlocking);
  for (int g = 0; g < b->ngroups && e == cudaSuccess; ++g)
    e = cudaStreamCreateWithFlags(&b->gstream[g], cudaStreamNonBlocking);
  for (int g = 0; g <= b->ngroups && e == cudaSuccess; ++g)
    e = cudaEventCreateWithFlags(&b->gev[g], cudaEventDisableTiming);
  for (int g = 0; g < b->ngroups; ++g)
    if (b->grp[g].svd_roles > 1) b->sample_branch = b->ngroups > 1;
  if (b->sample_branch && e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->sstream, cudaStreamNonBlocking);
  if (b->sample_branch && e == cudaSuccess) e = cudaEventCreateWithFlags(&b->sev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->dws, 0, bytes, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + oTiles, tiles.get(), (size_t)(count + b->ngroups) * 4, cudaMemcpyHostToDevice,
                        b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + oList, lists.get(), (size_t)count * 4, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    set_error("ircur_batch_create", e);
    ircur_batch_destroy(b);
    return IRCUR_ECUDA;
  }
  *out = b;
  return IRCUR_OK;
}

// One batched iteration, then the loop control.  One rank group: its core SVD
// and its panel pass (a programmatic dependent of the SVD) on s.  Several:
// every group's core SVD on a branch of its own, and the IRCUR-R look-ahead
// draws on one more, all forked from s and joined back; then every group's
// panel pass the same way.  (With the passes in the SVD branches, the pass
// blocks of the groups whose SVD ended first held the SMs that the other
// groups' SVDs waited for.)
static cudaError_t batch_iteration(ircur_batch* b, unsigned long long cond, cudaStream_t s, int par) {
  for (int g = 0; g < b->ngroups; ++g) b->grp[g].par = par;
  if (b->ngroups == 1) {
    cudaError_t e = launch_batch_group(b->grp[0], b->grpR[0], s);
    if (e != cudaSuccess) return e;
  } else {
    const int ng = b->ngroups;
    cudaError_t e = cudaEventRecord(b->gev[ng], s);
    if (e == cudaSuccess && b->sample_branch) {
      e = cudaStreamWaitEvent(b->sstream, b->gev[ng], 0);
      if (e == cudaSuccess) e = launch_sample_ahead_batch(b->ds, b->count, b->sstream);
      if (e == cudaSuccess) e = cudaEventRecord(b->sev, b->sstream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->sev, 0);
    }
    for (int g = 0; g < ng && e == cudaSuccess; ++g) {
      BatchLaunch bl = b->grp[g];
      if (b->sample_branch) bl.svd_roles = 1;
      e = cudaStreamWaitEvent(b->gstream[g], b->gev[ng], 0);
      if (e == cudaSuccess) e = launch_svd_batch(bl, b->grpR[g], b->gstream[g]);
      if (e == cudaSuccess) e = cudaEventRecord(b->gev[g], b->gstream[g]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->gev[g], 0);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->gev[ng], s);
    for (int g = 0; g < ng && e == cudaSuccess; ++g) {
      e = cudaStreamWaitEvent(b->gstream[g], b->gev[ng], 0);
      if (e == cudaSuccess) e = launch_batch_pass(b->grp[g], b->grpR[g], b->gstream[g]);
      if (e == cudaSuccess) e = cudaEventRecord(b->gev[g], b->gstream[g]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->gev[g], 0);
    }
    if (e != cudaSuccess) return e;
  }
  return launch_batch_check(b->ds, b->count, cond, b->any_active, s);
}

extern "C" ircur_ctx* ircur_batch_instance(ircur_batch* b, int32_t i) {
  if (!b || i < 0 || i >= b->count) return nullptr;
  return b->inst[i];
}

// Upload the descriptors the prologues left in each instance (no graph
// condition of their own: the loop-control kernel owns the batch's).
static ircur_status batch_upload_descs(ircur_batch* b) {
  for (int q = 0; q < b->count; ++q) {
    b->hdesc[q] = b->inst[b->order[q]]->desc;
    b->hdesc[q].cond = 0;
  }
  IRCUR_CK(cudaMemcpyAsync(b->ds, b->hdesc, (size_t)b->count * sizeof(IterDesc), cudaMemcpyHostToDevice,
                           b->stream));
  return IRCUR_OK;
}

static ircur_status batch_abort_capture(ircur_batch* b, cudaStream_t s, ircur_status st) {
  cudaGraph_t g = nullptr;
  cudaStreamEndCapture(s, &g);
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  batch_reset_graph(b);
  return st;
}

// One graph for a whole batch solve: every instance's prologue, the
// conditional while-node running the batched iteration, and the copies of the
// instances' states to pinned host memory.
static ircur_status batch_build_graph(ircur_batch* b, const float* const* D, const int64_t* ldD) {
  batch_reset_graph(b);
  cudaStream_t cs = b->capture_stream;
  IRCUR_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  for (int i = 0; i < b->count; ++i) {
    ircur_status ps = solve_prologue(b->inst[i], D[i], ldD[i], nullptr, nullptr, cs);
    if (ps != IRCUR_OK) return batch_abort_capture(b, cs, ps);
  }
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, &deps, nullptr, &ndeps);
  cudaGraphConditionalHandle h;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    set_error("batch graph: conditional handle", e);
    return batch_abort_capture(b, cs, IRCUR_ECUDA);
  }
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams* cp = reinterpret_cast<cudaGraphNodeParams*>(raw);
  cp->type = cudaGraphNodeTypeConditional;
  cp->conditional.handle = h;
  cp->conditional.type = cudaGraphCondTypeWhile;
  cp->conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, cp);
  if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) {
    set_error("batch graph: while node", e);
    return batch_abort_capture(b, cs, IRCUR_ECUDA);
  }
  e = cudaStreamBeginCaptureToGraph(b->body_stream, cp->conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) {
    set_error("batch graph: body capture", e);
    return batch_abort_capture(b, cs, IRCUR_ECUDA);
  }
  cudaError_t le = cudaSuccess;
  for (int u = 0; u < kGraphUnroll && le == cudaSuccess; ++u)
    le = batch_iteration(b, (unsigned long long)h, b->body_stream, u & 1);
  cudaGraph_t body = nullptr;
  cudaError_t be = cudaStreamEndCapture(b->body_stream, &body);
  if (le != cudaSuccess || be != cudaSuccess) {
    set_error("batch graph: iteration", le != cudaSuccess ? le : be);
    return batch_abort_capture(b, cs, IRCUR_ECUDA);
  }
  for (int i = 0; i < b->count; ++i) {
    e = cudaMemcpyAsync(b->hstates + b->pos[i], b->inst[i]->st, sizeof(State), cudaMemcpyDeviceToHost, cs);
    if (e != cudaSuccess) {
      set_error("batch graph: state copy", e);
      return batch_abort_capture(b, cs, IRCUR_ECUDA);
    }
  }
  e = cudaStreamEndCapture(cs, &b->graph);
  if (e != cudaSuccess) {
    set_error("batch graph: end capture", e);
    batch_reset_graph(b);
    return IRCUR_ECUDA;
  }
  IRCUR_CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
  ircur_status us = batch_upload_descs(b);
  if (us != IRCUR_OK) {
    batch_reset_graph(b);
    return us;
  }
  for (int i = 0; i < b->count; ++i) {
    b->graph_D[i] = D[i];
    b->graph_ld[i] = ldD[i];
  }
  return IRCUR_OK;
}

extern "C" ircur_status ircur_batch_solve(ircur_batch* b, const float* const* D, const int64_t* ldD,
                                          ircur_result* out) {
  if (!b || !D || !ldD || !out) return IRCUR_EINVAL;
  for (int i = 0; i < b->count; ++i) {
    if (!D[i] || ldD[i] < b->inst[i]->p.n2 || (reinterpret_cast<uintptr_t>(D[i]) & 3)) return IRCUR_EINVAL;
    b->inst[i]->solved = 0;
  }
  cudaStream_t s = b->stream;
  if (use_graph()) {
    bool same = b->exec != nullptr;
    for (int i = 0; same && i < b->count; ++i) same = b->graph_D[i] == D[i] && b->graph_ld[i] == ldD[i];
    if (!same) {
      ircur_status bs = batch_build_graph(b, D, ldD);
      if (bs != IRCUR_OK) return bs;
    }
    IRCUR_CK(cudaGraphLaunch(b->exec, s));
  } else {
    for (int i = 0; i < b->count; ++i) {
      ircur_status ps = solve_prologue(b->inst[i], D[i], ldD[i], nullptr, nullptr, s);
      if (ps != IRCUR_OK) return ps;
    }
    ircur_status us = batch_upload_descs(b);
    if (us != IRCUR_OK) return us;
    int active = 1;
    for (int it = 0; it < b->max_iter && active; ++it) {
      IRCUR_CK(batch_iteration(b, 0ull, s, it & 1));
      if ((it & 3) == 3) {
        IRCUR_CK(cudaMemcpyAsync(&active, b->any_active, sizeof(int), cudaMemcpyDeviceToHost, s));
        IRCUR_CK(cudaStreamSynchronize(s));
      }
    }
    for (int i = 0; i < b->count; ++i)
      IRCUR_CK(cudaMemcpyAsync(b->hstates + b->pos[i], b->inst[i]->st, sizeof(State), cudaMemcpyDeviceToHost, s));
  }
  IRCUR_CK(cudaStreamSynchronize(s));
  ircur_status first = IRCUR_OK;
  for (int i = 0; i < b->count; ++i) {
    b->inst[i]->host_state = b->hstates[b->pos[i]];
    const ircur_status si = solve_epilogue(b->inst[i], &out[i]);
    if (si != IRCUR_OK && first == IRCUR_OK) first = si;
  }
  return first;
}

// ---------------------------------------------------------------------------
// Autotuning of the panel-pass launch shape: whole solves timed with CUDA
// events for each candidate (resident blocks per SM, one or two tile buffers);
// the fastest stays in the context (or batch).

static int device_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = kNumSMsHint;
  return n;
}

struct TuneCand {
  int grid, single;
};

// svd_sms: SMs the core SVD holds while the pass kernel's blocks start (its
// programmatic dependents); one block fewer fits on each of them, so the
// largest grid is also tried without those blocks (0: not tried).
static int tune_candidates(int total, int resident2, int resident1, int sms, int svd_sms, TuneCand* out) {
  int n = 0;
  auto add = [&](int grid, int single) {
    if (grid > total) grid = total;
    if (grid < 1) return;
    for (int q = 0; q < n; ++q)
      if (out[q].grid == grid && out[q].single == single) return;
    if (n < IRCUR_TUNE_MAX) out[n++] = TuneCand{grid, single};
  };
  const int per2 = resident2 / sms, per1 = resident1 / sms;
  if (svd_sms > 0 && per2 >= 2) add(per2 * sms - svd_sms, 0);
  for (int k = per2; k >= 1; --k) add(k * sms, 0);
  if (per1 > per2) add(per1 * sms, 1);
  add(total, 0);  // one block per tile (blocks beyond the resident ones queue)
  return n;
}

static float median3(float* v, int n) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && v[j] < v[j - 1]; --j) {
      const float t = v[j];
      v[j] = v[j - 1];
      v[j - 1] = t;
    }
  return v[n / 2];
}

extern "C" ircur_status ircur_autotune(ircur_ctx* c, const float* D, int64_t ldD, int32_t reps,
                                       ircur_tune_result* out) {
  if (!c || !D || !out) return IRCUR_EINVAL;
  if (reps < 1) reps = 3;
  if (reps > 16) reps = 16;
  memset(out, 0, sizeof(*out));
  const int total = c->desc.nRowTiles + c->desc.nColTiles;
  const int sms = device_sms();
  IterDesc probe = c->desc;
  probe.passSingleBuf = 0;
  const int res2 = pass_resident_blocks(probe, c->Rpad);
  probe.passSingleBuf = 1;
  const int res1 = pass_resident_blocks(probe, c->Rpad);
  TuneCand cand[IRCUR_TUNE_MAX];
  const int nc = tune_candidates(total, res2, res1, sms, c->desc.svdNC, cand);
  cudaEvent_t e0, e1;
  IRCUR_CK(cudaEventCreate(&e0));
  IRCUR_CK(cudaEventCreate(&e1));
  ircur_status st = IRCUR_OK;
  int best = 0;
  for (int q = 0; q < nc && st == IRCUR_OK; ++q) {
    c->desc.passGrid = cand[q].grid;
    c->desc.passSingleBuf = cand[q].single;
    reset_graph(c);
    ircur_result r;
    st = ircur_solve(c, D, ldD, nullptr, nullptr, &r);  // warm-up (records the graph)
    float t[16];
    for (int k = 0; k < reps && st == IRCUR_OK; ++k) {
      cudaEventRecord(e0, c->stream);
      st = ircur_solve(c, D, ldD, nullptr, nullptr, &r);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t[k], e0, e1);
    }
    if (st != IRCUR_OK) break;
    out->grid[q] = cand[q].grid;
    out->single_buffer[q] = cand[q].single;
    out->ms[q] = median3(t, reps);
    if (out->ms[q] < out->ms[best]) best = q;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out->count = nc;
  out->chosen = best;
  c->desc.passGrid = nc > 0 ? cand[best].grid : 0;
  c->desc.passSingleBuf = nc > 0 ? cand[best].single : 0;
  reset_graph(c);
  return st;
}

extern "C" ircur_status ircur_batch_autotune(ircur_batch* b, const float* const* D, const int64_t* ldD, int32_t reps,
                                             ircur_tune_result* out) {
  if (!b || !D || !ldD || !out) return IRCUR_EINVAL;
  if (reps < 1) reps = 3;
  if (reps > 16) reps = 16;
  memset(out, 0, sizeof(*out));
  const int sms = device_sms();
  // per group: resident blocks with two tile buffers and with one
  int per2[kMaxRankGroups], per1[kMaxRankGroups], nbuf2[kMaxRankGroups], nbuf1[kMaxRankGroups];
  size_t smem2[kMaxRankGroups], smem1[kMaxRankGroups];
  int maxper = 1, total = 0;
  for (int g = 0; g < b->ngroups; ++g) {
    BatchLaunch& bl = b->grp[g];
    const int mm = bl.pass_mmax, R = b->grpR[g];
    bl.pass_grid = 0;
    smem2[g] = pass_smem_bytes(mm, mm, R, &nbuf2[g], false, false);
    smem1[g] = pass_smem_bytes(mm, mm, R, &nbuf1[g], false, true);
    bl.pass_smem = smem2[g];
    bl.pass_nbuf = nbuf2[g];
    per2[g] = pass_batch_resident_blocks(bl, R) / sms;
    bl.pass_smem = smem1[g];
    bl.pass_nbuf = nbuf1[g];
    per1[g] = pass_batch_resident_blocks(bl, R) / sms;
    if (per1[g] > maxper) maxper = per1[g];
    total += bl.total_tiles;
  }
  // candidates: k resident blocks per SM (capped per group) with two or one
  // tile buffers, or one block per tile (k = 0).  (Grids in proportion to each
  // group's share of the tiles, so that the groups' concurrent pass kernels
  // split the GPU, measured 1.5-2.3x slower on the 64-instance batch.)
  TuneCand cand[IRCUR_TUNE_MAX];
  int nc = 0;
  for (int k = 1; k <= maxper && nc < IRCUR_TUNE_MAX - 1; ++k) {
    cand[nc++] = TuneCand{k, 0};
    if (nc < IRCUR_TUNE_MAX - 1) cand[nc++] = TuneCand{k, 1};
  }
  cand[nc++] = TuneCand{0, 0};
  auto apply = [&](const TuneCand& tc) {
    for (int g = 0; g < b->ngroups; ++g) {
      BatchLaunch& bl = b->grp[g];
      const int per = tc.single ? per1[g] : per2[g];
      bl.pass_smem = tc.single ? smem1[g] : smem2[g];
      bl.pass_nbuf = tc.single ? nbuf1[g] : nbuf2[g];
      const int k = tc.grid == 0 ? 0 : (tc.grid < per ? tc.grid : (per > 0 ? per : 1));
      bl.pass_grid = k == 0 ? bl.total_tiles : k * sms;
    }
    batch_reset_graph(b);
  };
  ircur_result* res = new (std::nothrow) ircur_result[b->count];
  if (!res) return IRCUR_ENOMEM;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    delete[] res;
    return IRCUR_ECUDA;
  }
  ircur_status st = IRCUR_OK;
  int best = 0;
  for (int q = 0; q < nc && st == IRCUR_OK; ++q) {
    apply(cand[q]);
    st = ircur_batch_solve(b, D, ldD, res);
    float t[16];
    for (int k = 0; k < reps && st == IRCUR_OK; ++k) {
      cudaEventRecord(e0, b->stream);
      st = ircur_batch_solve(b, D, ldD, res);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t[k], e0, e1);
    }
    if (st != IRCUR_OK) break;
    out->grid[q] = cand[q].grid == 0 ? total : cand[q].grid * sms;
    out->single_buffer[q] = cand[q].single;
    out->ms[q] = median3(t, reps);
    if (out->ms[q] < out->ms[best]) best = q;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  delete[] res;
  out->count = nc;
  out->chosen = best;
  if (nc > 0) apply(cand[best]);
  return st;
}

