// ircur_solve_noalloc: a one-shot IRCUR-F solve that allocates nothing.
//
// Some callers may not call cudaMalloc at all: a process whose memory pool has
// already reserved the device memory it is allowed to use (a fresh driver
// allocation would fail or fragment it), or a latency-bound loop in which
// cudaMalloc's implicit device synchronisation and unbounded latency are not
// acceptable.  For them this entry point runs the same kernels as ircur_solve
// with its workspace carved from one file-scope device array of fixed size,
// which every GPU that loads the library holds until the process exits.
//
// Limits (the array is sized for them): IRCUR-F only (IRCUR-R keeps a
// transposed copy of D, which would not be modest); n1, n2 <= 2048;
// |I|, |J| <= 192; r <= 8; max_iter <= 256.
//
// Every call shares the array and it keeps the last call's contents; each call
// clears what must start at zero.  Calls that overlap on the GPU (two streams,
// or two host threads) race on the array and must not be issued.
#include <math.h>
#include <string.h>

#include <mutex>

#include "ircur.h"
#include "ircur_internal.cuh"

using namespace ircur;

namespace {

constexpr int64_t kNaMaxN = 2048;
constexpr int kNaMaxM = 192;
constexpr int kNaMaxR = 8;  // padded rank
constexpr int kNaMaxIter = 256;

constexpr size_t na_piece(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

constexpr size_t kNaBytes =
    2 * na_piece((size_t)kNaMaxM * 4) +                                  // I, J (one draw)
    na_piece((size_t)kNaMaxM * kNaMaxN * 4) +                            // D(I,:)
    na_piece((size_t)kNaMaxM * kNaMaxN * 4) +                            // D(:,J)^T
    4 * na_piece((size_t)kNaMaxN * kNaMaxR * 4) +                        // A[2], B[2]
    na_piece((size_t)kNaMaxM * kNaMaxM * 4) +                            // D(I,J)
    2 * na_piece((size_t)kNaMaxN * 4) +                                  // index maps
    4 * na_piece((size_t)kNaMaxM * kNaMaxR * 4) +                        // A_k(I,:), B_k(:,J)^T by parity
    3 * na_piece((size_t)kNaMaxM * kNaMaxR * 4) +                        // W, V, Vs
    na_piece((size_t)kNaMaxR * 4) + na_piece((size_t)kNaMaxR * kNaMaxR * 4) +  // sigma, T
    na_piece((size_t)((kNaMaxN + kPanelCols - 1) / kPanelCols * 2) * 2 * 8) +  // partials
    na_piece((size_t)kNaMaxIter * 8) +                                   // e_k history
    na_piece(sizeof(State));

}  // namespace

// The workspace of ircur_solve_noalloc (3.5 MB), 256-byte aligned.
static __device__ __align__(256) unsigned char g_noalloc_ws[kNaBytes];

namespace {

std::mutex g_na_mu;
void* g_na_addr[256];  // device address of g_noalloc_ws, per device ordinal

}  // namespace

extern "C" ircur_status ircur_solve_noalloc(const ircur_params* params, const float* D, int64_t ldD, float* A,
                                            float* B, ircur_result* out, void* stream) {
  if (!params || !D || !A || !B || !out) return IRCUR_EINVAL;
  ircur_params p = *params;
  if (p.n1 < 1 || p.n2 < 1 || p.r < 1) return IRCUR_EINVAL;
  if (p.nI == 0) p.nI = (int)fmin((double)p.n1, ceil(4.0 * p.r * log((double)p.n1)));
  if (p.nJ == 0) p.nJ = (int)fmin((double)p.n2, ceil(4.0 * p.r * log((double)p.n2)));
  if (p.nI < p.r || p.nJ < p.r || p.nI > p.n1 || p.nJ > p.n2) return IRCUR_EINVAL;
  if (!(p.gamma > 0.0 && p.gamma < 1.0) || !(p.tol > 0.0) || p.max_iter < 1) return IRCUR_EINVAL;
  if (p.resample != 0 || p.precision != 0) return IRCUR_EINVAL;
  if (p.svd_form != IRCUR_SVD_CLUSTER && p.svd_form != IRCUR_SVD_ONE_CTA) return IRCUR_EINVAL;
  if (!(p.zeta0 == p.zeta0)) return IRCUR_EINVAL;
  // sizes beyond the fixed workspace
  if (p.n1 > kNaMaxN || p.n2 > kNaMaxN || p.nI > kNaMaxM || p.nJ > kNaMaxM || pad_rank(p.r) > kNaMaxR ||
      p.max_iter > kNaMaxIter)
    return IRCUR_EINVAL;
  if (ldD < p.n2 || (reinterpret_cast<uintptr_t>(D) & 3)) return IRCUR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // device address of the workspace, looked up once per device (the first
  // call on each device, with that device current).  The address stays valid
  // for the life of the device's primary context: a cudaDeviceReset after the
  // first call is not supported (the module may be reloaded elsewhere).
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) return IRCUR_ECUDA;
  unsigned char* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_ws);
      if (e != cudaSuccess || !ptr) return IRCUR_ECUDA;
      g_na_addr[dev] = ptr;
    }
    ws = static_cast<unsigned char*>(g_na_addr[dev]);
  }

  const int R = pad_rank(p.r);
  const int64_t n1 = p.n1, n2 = p.n2;
  const int64_t ldDc = (p.nJ + 3) & ~3ll;
  IterDesc d;
  memset(&d, 0, sizeof(d));
  d.svdNC = svd_cluster_size(p.nI, p.nJ, R, p.svd_form);
  if (d.svdNC == 0) return IRCUR_EINVAL;
  d.nRowTiles = (int)((n2 + kPanelCols - 1) / kPanelCols);
  d.nColTiles = (int)((n1 + kPanelCols - 1) / kPanelCols);
  const int64_t ldPr = (n2 + 3) & ~3ll, ldPc = (n1 + 3) & ~3ll;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* q = ws + off;
    off += na_piece(bytes);
    return q;
  };
  int* I = reinterpret_cast<int*>(take((size_t)p.nI * 4));
  int* J = reinterpret_cast<int*>(take((size_t)p.nJ * 4));
  float* Prow = reinterpret_cast<float*>(take((size_t)p.nI * ldPr * 4));
  float* PcolT = reinterpret_cast<float*>(take((size_t)p.nJ * ldPc * 4));
  float* Ab[2];
  float* Bb[2];
  Ab[0] = reinterpret_cast<float*>(take((size_t)n1 * R * 4));
  Ab[1] = reinterpret_cast<float*>(take((size_t)n1 * R * 4));
  Bb[0] = reinterpret_cast<float*>(take((size_t)R * n2 * 4));
  Bb[1] = reinterpret_cast<float*>(take((size_t)R * n2 * 4));
  float* Dc = reinterpret_cast<float*>(take((size_t)p.nI * ldDc * 4));
  unsigned* posI = reinterpret_cast<unsigned*>(take((size_t)n1 * 4));
  unsigned* posJ = reinterpret_cast<unsigned*>(take((size_t)n2 * 4));
  float* AIc[2];
  float* BJc[2];
  for (int q = 0; q < 2; ++q) {
    AIc[q] = reinterpret_cast<float*>(take((size_t)p.nI * R * 4));
    BJc[q] = reinterpret_cast<float*>(take((size_t)p.nJ * R * 4));
  }
  float* W = reinterpret_cast<float*>(take((size_t)p.nI * R * 4));
  float* V = reinterpret_cast<float*>(take((size_t)p.nJ * R * 4));
  float* Vs = reinterpret_cast<float*>(take((size_t)p.nJ * R * 4));
  float* sigma = reinterpret_cast<float*>(take((size_t)R * 4));
  float* Tm = reinterpret_cast<float*>(take((size_t)R * R * 4));
  float* partials = reinterpret_cast<float*>(take((size_t)(d.nRowTiles + d.nColTiles) * 2 * 4));
  double* errs = reinterpret_cast<double*>(take((size_t)p.max_iter * 8));
  State* st = reinterpret_cast<State*>(take(sizeof(State)));
  if (off > kNaBytes) return IRCUR_EINVAL;  // cannot happen within the limits above

  d.n1 = n1;
  d.n2 = n2;
  d.r = p.r;
  d.nI = p.nI;
  d.nJ = p.nJ;
  d.max_iter = p.max_iter;
  d.resample = 0;
  d.gamma = p.gamma;
  d.tol = p.tol;
  d.D = D;
  d.ldD = ldD;
  d.rowSrc = Prow;
  d.rowLd = ldPr;
  d.colSrc = PcolT;
  d.colLd = ldPc;
  d.Prow = Prow;
  d.ldPr = ldPr;
  d.PcolT = PcolT;
  d.ldPc = ldPc;
  d.I_all = I;
  d.J_all = J;
  d.A[0] = Ab[0];
  d.A[1] = Ab[1];
  d.B[0] = Bb[0];
  d.B[1] = Bb[1];
  d.Dc[0] = d.Dc[1] = Dc;
  d.posI[0] = d.posI[1] = posI;
  d.posJ[0] = d.posJ[1] = posJ;
  for (int q = 0; q < 2; ++q) {
    d.AI[q] = AIc[q];
    d.BJt[q] = BJc[q];
  }
  d.ldDc = ldDc;
  d.W = W;
  d.V = V;
  d.Vs = Vs;
  d.sigma = sigma;
  d.Tm = Tm;
  d.partials = partials;
  d.errs = errs;
  d.st = st;
  d.rowBulk = 1;
  d.colBulk = 1;
  d.svdMaxSteps = 500;
  d.spinLimit = kSpinLimit;
  d.sampleAhead = 0;
  d.cond = 0;
  d.seed = p.seed;

#define NA_CK(call)                        \
  do {                                     \
    if ((call) != cudaSuccess) return IRCUR_ECUDA; \
  } while (0)

  // what must start at zero: the whole carved region (factors A_0 = B_0 = 0,
  // the core's padding columns, the state's counters)
  NA_CK(cudaMemsetAsync(ws, 0, off, s));
  NA_CK(launch_setup(d, p.zeta0 > 0 ? p.zeta0 : 0.0, s));
  unsigned* maps_I[2] = {posI, posI};
  unsigned* maps_J[2] = {posJ, posJ};
  NA_CK(launch_sample(p.seed, 0, 1, n1, n2, p.nI, p.nJ, I, J, -1, s, maps_I, maps_J));
  if (!(p.zeta0 > 0)) {
    NA_CK(launch_maxabs(D, n1, n2, ldD, st, s));
    NA_CK(launch_finalize_zeta(st, s));
  }
  NA_CK(launch_gather(d, s));
  NA_CK(launch_gather_core(d, 0, 0, s));
  State h;
  memset(&h, 0, sizeof(h));
  for (int it = 0; it < p.max_iter; ++it) {
    d.par = it & 1;
    NA_CK(launch_iteration(d, R, s));
    if ((it & 3) == 3 || it + 1 == p.max_iter) {
      NA_CK(cudaMemcpyAsync(&h, st, sizeof(State), cudaMemcpyDeviceToHost, s));
      NA_CK(cudaStreamSynchronize(s));
      if (h.done) break;
    }
  }
  const int K = h.k;
  NA_CK(cudaMemcpy2DAsync(A, (size_t)p.r * 4, Ab[K & 1], (size_t)R * 4, (size_t)p.r * 4, (size_t)n1,
                          cudaMemcpyDeviceToDevice, s));
  NA_CK(cudaMemcpyAsync(B, Bb[K & 1], (size_t)p.r * n2 * 4, cudaMemcpyDeviceToDevice, s));
  NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
  memset(out, 0, sizeof(*out));
  out->iters = h.k;
  out->converged = (h.k > 0 && h.e <= p.tol) ? 1 : 0;
  out->flags = h.flags;
  out->svd_steps = h.svd_steps;
  out->final_err = h.e;
  out->zeta0 = h.zeta0;
  out->zeta_next = h.zeta;
  if (h.status != 0) return (ircur_status)h.status;
  return IRCUR_OK;
}
