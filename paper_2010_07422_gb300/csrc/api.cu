// Host side of libircur: the extern "C" entry points declared in ircur.h,
// workspace management, and the CUDA graph that runs Alg. 1's loop on the
// device (a conditional while-node whose body is one iteration; the pass
// kernel's last block evaluates the stopping test of Sec. 3.3 and sets the
// node's condition, so no host round trip happens inside the loop).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

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
  float* AI;
  float* BJt;
  float* core;
  float* W;
  float* V;
  float* Vs;
  float* sigma;
  float* Tm;
  double* partials;
  double* errs;
  State* st;
  // graph cache
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  const float* graph_D;
  int64_t graph_ldD;
  int graph_sample_ahead;
  unsigned long long* graph_trace;
  unsigned long long* trace;  // kernel-span trace buffer (2 * 3 * max_iter), or null
  // last solve
  int solved;
  State host_state;
  // buffers of the host-memory entry point
  float* hD;
  float* hL;
  float* hS;
  IterDesc desc;
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
  if (pass_smem_bytes(q.nI, q.nJ, pad_rank(q.r)) > 227 * 1024) return IRCUR_ENOTSUP;
  {
    bool in_smem = false;
    if (svd_smem_bytes(q.nI, q.nJ, pad_rank(q.r), &in_smem) > 227 * 1024) return IRCUR_ENOTSUP;
  }
  if (!(q.gamma > 0.0 && q.gamma < 1.0)) return IRCUR_EINVAL;
  if (!(q.tol > 0.0)) return IRCUR_EINVAL;
  if (q.max_iter < 1) return IRCUR_EINVAL;
  if (q.resample != 0 && q.resample != 1) return IRCUR_EINVAL;
  if (q.precision != 0) return IRCUR_ENOTSUP;
  if (q.reserved != 0) return IRCUR_EINVAL;
  if (!(q.zeta0 == q.zeta0)) return IRCUR_EINVAL;
  *out = q;
  return IRCUR_OK;
}

extern "C" ircur_status ircur_create(const ircur_params* params, void* stream, ircur_ctx** out) {
  if (!out) return IRCUR_EINVAL;
  *out = nullptr;
  ircur_params p;
  ircur_status vs = validate_params(params, &p);
  if (vs != IRCUR_OK) return vs;
  if (strcmp(fault_mode(), "alloc") == 0) return IRCUR_ENOMEM;

  ircur_ctx* c = new (std::nothrow) ircur_ctx();
  if (!c) return IRCUR_ENOMEM;
  c->p = p;
  c->Rpad = pad_rank(p.r);
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  c->draws = p.resample ? p.max_iter : 1;
  const int R = c->Rpad;
  const int64_t n1 = p.n1, n2 = p.n2;
  c->ldPr = (n2 + 3) & ~3ll;
  c->ldPc = (n1 + 3) & ~3ll;
  c->ldDT = (n1 + 3) & ~3ll;

  // tile configuration of the pass kernel
  IterDesc& d = c->desc;
  memset(&d, 0, sizeof(d));
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
  const size_t oPr = p.resample ? 0 : take((size_t)p.nI * c->ldPr * 4);
  const size_t oPc = p.resample ? 0 : take((size_t)p.nJ * c->ldPc * 4);
  const size_t oDT = p.resample ? take((size_t)n2 * c->ldDT * 4) : 0;
  const size_t oA0 = take((size_t)n1 * R * 4), oA1 = take((size_t)n1 * R * 4);
  const size_t oB0 = take((size_t)R * n2 * 4), oB1 = take((size_t)R * n2 * 4);
  int ldCore = (p.nJ + 3) & ~3;
  if (((ldCore / 4) & 1) == 0) ldCore += 4;
  d.ldCore = ldCore;
  const size_t oCore = take((size_t)p.nI * ldCore * 4);
  const size_t oAI = take((size_t)p.nI * R * 4), oBJ = take((size_t)p.nJ * R * 4);
  const size_t oW = take((size_t)p.nI * R * 4), oV = take((size_t)p.nJ * R * 4), oVs = take((size_t)p.nJ * R * 4);
  const size_t oSig = take((size_t)R * 4);
  const size_t oTm = take((size_t)R * R * 4);
  const size_t oPart = take((size_t)(d.nRowTiles + d.nColTiles) * 2 * 8);
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
  c->Prow = p.resample ? nullptr : reinterpret_cast<float*>(base + oPr);
  c->PcolT = p.resample ? nullptr : reinterpret_cast<float*>(base + oPc);
  c->DT = p.resample ? reinterpret_cast<float*>(base + oDT) : nullptr;
  c->A[0] = reinterpret_cast<float*>(base + oA0);
  c->A[1] = reinterpret_cast<float*>(base + oA1);
  c->B[0] = reinterpret_cast<float*>(base + oB0);
  c->B[1] = reinterpret_cast<float*>(base + oB1);
  c->core = reinterpret_cast<float*>(base + oCore);
  c->AI = reinterpret_cast<float*>(base + oAI);
  c->BJt = reinterpret_cast<float*>(base + oBJ);
  c->W = reinterpret_cast<float*>(base + oW);
  c->V = reinterpret_cast<float*>(base + oV);
  c->Vs = reinterpret_cast<float*>(base + oVs);
  c->sigma = reinterpret_cast<float*>(base + oSig);
  c->Tm = reinterpret_cast<float*>(base + oTm);
  c->partials = reinterpret_cast<double*>(base + oPart);
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
  d.core = c->core;
  d.AI = c->AI;
  d.BJt = c->BJt;
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

extern "C" void ircur_destroy(ircur_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  reset_graph(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->trace) cudaFree(c->trace);
  if (c->hD) cudaFree(c->hD);
  if (c->hL) cudaFree(c->hL);
  if (c->hS) cudaFree(c->hS);
  if (c->ws) cudaFree(c->ws);
  delete c;
}

static bool use_graph() {
  const char* g = getenv("IRCUR_NO_GRAPH");
  return !(g && g[0] == '1');
}

// Build (or reuse) the graph: one conditional while-node whose body is one
// iteration (core, SVD, passes).  The body is recorded by stream capture on
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
  cudaError_t le = launch_iteration(d, c->Rpad, c->capture_stream);
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
  return IRCUR_OK;
}

static ircur_status read_state(ircur_ctx* c) {
  IRCUR_CK(cudaMemcpyAsync(&c->host_state, c->st, sizeof(State), cudaMemcpyDeviceToHost, c->stream));
  IRCUR_CK(cudaStreamSynchronize(c->stream));
  return IRCUR_OK;
}

extern "C" ircur_status ircur_solve(ircur_ctx* c, const float* D, int64_t ldD, const int32_t* idx_I,
                                    const int32_t* idx_J, ircur_result* out) {
  if (!c || !D || !out) return IRCUR_EINVAL;
  const ircur_params& p = c->p;
  if (ldD < p.n2 || (reinterpret_cast<uintptr_t>(D) & 3)) return IRCUR_EINVAL;
  if ((idx_I == nullptr) != (idx_J == nullptr)) return IRCUR_EINVAL;
  cudaStream_t s = c->stream;
  IterDesc d = c->desc;
  d.D = D;
  d.ldD = ldD;
  d.rowSrc = p.resample ? D : c->Prow;
  d.rowLd = p.resample ? ldD : c->ldPr;
  d.rowBulk = p.resample ? ((aligned16(D) && ldD % 4 == 0) ? 1 : 0) : 1;
  d.sampleAhead = (p.resample && !idx_I) ? 1 : 0;
  d.trace = c->trace;
  c->desc = d;
  if (c->trace) {
    const size_t half = (size_t)3 * p.max_iter * 8;
    IRCUR_CK(cudaMemsetAsync(c->trace, 0xFF, half, s));
    IRCUR_CK(cudaMemsetAsync(reinterpret_cast<char*>(c->trace) + half, 0, half, s));
  }

  const double zeta0 = p.zeta0 > 0 ? p.zeta0 : 0.0;
  IRCUR_CK(launch_setup(d, zeta0, s));
  if (idx_I) {
    IRCUR_CK(cudaMemcpyAsync(c->I_all, idx_I, (size_t)c->draws * p.nI * 4, cudaMemcpyDeviceToDevice, s));
    IRCUR_CK(cudaMemcpyAsync(c->J_all, idx_J, (size_t)c->draws * p.nJ * 4, cudaMemcpyDeviceToDevice, s));
    IRCUR_CK(launch_check_indices(c->I_all, c->draws, p.nI, p.n1, &c->st->status, s));
    IRCUR_CK(launch_check_indices(c->J_all, c->draws, p.nJ, p.n2, &c->st->status, s));
  } else {
    // draw 0 now; IRCUR-R draws k+1 alongside iteration k's core SVD
    IRCUR_CK(launch_sample(p.seed, 0, 1, p.n1, p.n2, p.nI, p.nJ, c->I_all, c->J_all, -1, s));
  }
  if (p.resample) {
    // D^T for the column panels, with max|D| and the NaN/Inf scan in the same pass
    IRCUR_CK(launch_transpose_maxabs(D, p.n1, p.n2, ldD, c->DT, c->ldDT, c->st, s));
  } else if (!(p.zeta0 > 0)) {
    IRCUR_CK(launch_maxabs(D, p.n1, p.n2, ldD, c->st, s));
  }
  if (!(p.zeta0 > 0)) IRCUR_CK(launch_finalize_zeta(c->st, s));
  if (!p.resample) IRCUR_CK(launch_gather(d, s));
  IRCUR_CK(cudaMemsetAsync(c->A[0], 0, (size_t)p.n1 * c->Rpad * 4, s));
  IRCUR_CK(cudaMemsetAsync(c->B[0], 0, (size_t)c->Rpad * p.n2 * 4, s));

  if (use_graph()) {
    if (!c->exec || c->graph_D != D || c->graph_ldD != ldD || c->graph_sample_ahead != d.sampleAhead ||
        c->graph_trace != d.trace) {
      ircur_status bs = build_graph(c, d);
      if (bs != IRCUR_OK) return bs;
    }
    IRCUR_CK(cudaGraphLaunch(c->exec, s));
  } else {
    // Host-driven loop (profiling and debugging: every kernel is a separate
    // launch).  The device flag is polled every few iterations.
    for (int it = 0; it < p.max_iter; ++it) {
      IRCUR_CK(launch_iteration(d, c->Rpad, s));
      if ((it & 3) == 3) {
        ircur_status rs = read_state(c);
        if (rs != IRCUR_OK) return rs;
        if (c->host_state.done) break;
      }
    }
  }
  ircur_status rs = read_state(c);
  if (rs != IRCUR_OK) return rs;
  const State& h = c->host_state;
  c->solved = 1;
  memset(out, 0, sizeof(*out));
  out->iters = h.k;
  out->converged = (h.k > 0 && h.e <= p.tol) ? 1 : 0;
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

extern "C" ircur_status ircur_solve_host(ircur_ctx* c, const float* D_host, float* L_host, float* S_host,
                                         ircur_result* out) {
  if (!c || !D_host || !L_host || !out) return IRCUR_EINVAL;
  const ircur_params& p = c->p;
  const size_t bytes = (size_t)p.n1 * p.n2 * 4;
  if (!c->hD) {
    cudaError_t e = cudaMalloc(&c->hD, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->hL, bytes);
    if (e != cudaSuccess) {
      set_error("cudaMalloc(host-path buffers)", e);
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
  IRCUR_CK(cudaMemcpyAsync(c->hD, D_host, bytes, cudaMemcpyHostToDevice, c->stream));
  ircur_status s = ircur_solve(c, c->hD, p.n2, nullptr, nullptr, out);
  if (s != IRCUR_OK) return s;
  s = ircur_reconstruct(c, c->hD, p.n2, c->hL, p.n2, S_host ? c->hS : nullptr, p.n2);
  if (s != IRCUR_OK) return s;
  IRCUR_CK(cudaMemcpyAsync(L_host, c->hL, bytes, cudaMemcpyDeviceToHost, c->stream));
  if (S_host) IRCUR_CK(cudaMemcpyAsync(S_host, c->hS, bytes, cudaMemcpyDeviceToHost, c->stream));
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
    cudaError_t e = cudaMalloc(&c->trace, (size_t)2 * 3 * c->p.max_iter * 8);
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
  const int n = 3 * c->p.max_iter;
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
  for (int q = 0; q < 3 * K; ++q)
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
