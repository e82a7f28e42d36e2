"""Python binding of libircur (ctypes): the C-ABI entry points under the same
names, plus a small convenience layer over torch tensors.

Argument marshalling only: every step of IRCUR runs in the CUDA library.  If
the library is missing the first call raises; there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libircur.so")

IRCUR_OK, IRCUR_EINVAL, IRCUR_ENOMEM, IRCUR_ECUDA = 0, 1, 2, 3
IRCUR_ESVD_NOCONV, IRCUR_ETIMEOUT, IRCUR_ESTATE, IRCUR_ENOTSUP = 4, 5, 6, 7
IRCUR_FLAG_WRANK, IRCUR_FLAG_SVD_NOCONV, IRCUR_FLAG_SVD_GAP = 1, 2, 4
IRCUR_MAX_RANK = 20
IRCUR_PRECISION_FP32, IRCUR_PRECISION_BF16_PANELS = 0, 1
IRCUR_SVD_CLUSTER, IRCUR_SVD_ONE_CTA, IRCUR_SVD_CLUSTER8 = 0, 1, 2

EXPORTED = (
    "ircur_create", "ircur_destroy", "ircur_solve", "ircur_get_factors", "ircur_get_indices",
    "ircur_get_errors", "ircur_reconstruct", "ircur_solve_host", "ircur_sample_indices",
    "ircur_status_string", "ircur_last_error_string", "ircur_solve_noalloc", "ircur_set_trace",
    "ircur_get_trace", "ircur_get_cur", "ircur_batch_create", "ircur_batch_destroy", "ircur_batch_solve",
    "ircur_batch_instance", "ircur_set_record", "ircur_backward", "ircur_autotune", "ircur_batch_autotune",
    "ircur_get_svd", "ircur_stream_columns", "ircur_get_launch_shape",
)


class ircur_params(C.Structure):
    _fields_ = [("n1", C.c_int64), ("n2", C.c_int64), ("r", C.c_int32), ("nI", C.c_int32),
                ("nJ", C.c_int32), ("zeta0", C.c_double), ("gamma", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int32), ("resample", C.c_int32), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("svd_form", C.c_int32)]


class ircur_result(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("flags", C.c_uint32),
                ("svd_steps", C.c_int32), ("final_err", C.c_double), ("zeta0", C.c_double),
                ("zeta_next", C.c_double)]


class ircur_tune_result(C.Structure):
    _fields_ = [("count", C.c_int32), ("chosen", C.c_int32), ("grid", C.c_int32 * 8),
                ("single_buffer", C.c_int32 * 8), ("ms", C.c_float * 8)]

    def as_dict(self):
        return {"chosen": self.chosen,
                "candidates": [{"grid": self.grid[i], "single_buffer": self.single_buffer[i],
                                "ms": self.ms[i]} for i in range(self.count)]}


class IrcurError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        lib = _lib()
        msg = lib.ircur_status_string(status).decode()
        cuda = lib.ircur_last_error_string().decode()
        super().__init__(f"{where}: {msg}" + (f" [{cuda}]" if cuda and status == IRCUR_ECUDA else ""))


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the IRCUR path has no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        P, I64, I32, U64 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint64
        lib.ircur_create.argtypes = [C.POINTER(ircur_params), P, C.POINTER(P)]
        lib.ircur_destroy.argtypes = [P]
        lib.ircur_destroy.restype = None
        lib.ircur_solve.argtypes = [P, P, I64, P, P, C.POINTER(ircur_result)]
        lib.ircur_get_factors.argtypes = [P, P, P]
        lib.ircur_get_indices.argtypes = [P, P, P, P]
        lib.ircur_get_errors.argtypes = [P, C.POINTER(C.c_double), C.POINTER(I32)]
        lib.ircur_get_launch_shape.argtypes = [P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)]
        lib.ircur_reconstruct.argtypes = [P, P, I64, P, I64, P, I64]
        lib.ircur_solve_host.argtypes = [P, P, P, P, C.POINTER(ircur_result)]
        lib.ircur_sample_indices.argtypes = [U64, I32, I32, I64, I32, P, P]
        lib.ircur_solve_noalloc.argtypes = [C.POINTER(ircur_params), P, I64, P, P, C.POINTER(ircur_result), P]
        lib.ircur_set_trace.argtypes = [P, I32]
        lib.ircur_get_cur.argtypes = [P, P, I64, P, P, P]
        lib.ircur_get_trace.argtypes = [P, C.POINTER(C.c_double), C.POINTER(I32)]
        lib.ircur_batch_create.argtypes = [C.POINTER(ircur_params), I32, P, C.POINTER(P)]
        lib.ircur_batch_destroy.argtypes = [P]
        lib.ircur_batch_destroy.restype = None
        lib.ircur_batch_solve.argtypes = [P, C.POINTER(P), C.POINTER(I64), C.POINTER(ircur_result)]
        lib.ircur_batch_instance.argtypes = [P, I32]
        lib.ircur_batch_instance.restype = P
        lib.ircur_set_record.argtypes = [P, I32]
        lib.ircur_backward.argtypes = [P, P, I64, P, I64, P, I64, P, I64]
        lib.ircur_get_svd.argtypes = [P, P, P, P]
        lib.ircur_stream_columns.argtypes = [P, P, I64, I64, I32, P, I64, P, I64]
        lib.ircur_autotune.argtypes = [P, P, I64, I32, C.POINTER(ircur_tune_result)]
        lib.ircur_batch_autotune.argtypes = [P, C.POINTER(P), C.POINTER(I64), I32, C.POINTER(ircur_tune_result)]
        lib.ircur_status_string.argtypes = [C.c_int]
        lib.ircur_status_string.restype = C.c_char_p
        lib.ircur_last_error_string.argtypes = []
        lib.ircur_last_error_string.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("ircur_destroy", "ircur_status_string", "ircur_last_error_string",
                            "ircur_batch_destroy", "ircur_batch_instance"):
                getattr(lib, name).restype = C.c_int
        _LIB = lib
    return _LIB


def _check(status, where):
    if status != IRCUR_OK:
        raise IrcurError(status, where)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_handle(device=None):
    import torch
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def sample_size(c, r, n):
    """|I| = ceil(c r ln n), capped at n (Sec. 3.5)."""
    return int(min(n, math.ceil(c * r * math.log(n))))


# ---------------------------------------------------------------- raw entry points
def ircur_create(params: ircur_params, stream=None):
    ctx = C.c_void_p()
    _check(_lib().ircur_create(C.byref(params), stream, C.byref(ctx)), "ircur_create")
    return ctx


def ircur_destroy(ctx):
    _lib().ircur_destroy(ctx)


def ircur_solve(ctx, D, ldD, idx_I=None, idx_J=None):
    res = ircur_result()
    _check(_lib().ircur_solve(ctx, _ptr(D), ldD, _ptr(idx_I), _ptr(idx_J), C.byref(res)), "ircur_solve")
    return res


def ircur_get_factors(ctx, A=None, B=None):
    _check(_lib().ircur_get_factors(ctx, _ptr(A), _ptr(B)), "ircur_get_factors")


def ircur_get_indices(ctx, I=None, J=None, sigma=None):
    _check(_lib().ircur_get_indices(ctx, _ptr(I), _ptr(J), _ptr(sigma)), "ircur_get_indices")


def ircur_get_errors(ctx, max_iter):
    buf = (C.c_double * max_iter)()
    cnt = C.c_int32()
    _check(_lib().ircur_get_errors(ctx, buf, C.byref(cnt)), "ircur_get_errors")
    return list(buf[: cnt.value])


def ircur_get_launch_shape(ctx):
    """(svd_ctas, pass_blocks, pass_bufs) of the context's iterations."""
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib().ircur_get_launch_shape(ctx, C.byref(a), C.byref(b), C.byref(c)), "ircur_get_launch_shape")
    return a.value, b.value, c.value


def ircur_reconstruct(ctx, D, ldD, L, ldL, S=None, ldS=0):
    _check(_lib().ircur_reconstruct(ctx, _ptr(D), ldD, _ptr(L), ldL, _ptr(S), ldS), "ircur_reconstruct")


def ircur_stream_columns(ctx, Dnew, ldDn, ncols, iters, L, ldL, S=None, ldS=0):
    _check(_lib().ircur_stream_columns(ctx, _ptr(Dnew), ldDn, ncols, iters, _ptr(L), ldL, _ptr(S), ldS),
           "ircur_stream_columns")


def ircur_solve_host(ctx, D_host, L_host, S_host=None):
    """D_host, L_host, S_host: C-contiguous float32 numpy arrays or pinned CPU tensors."""
    def hp(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return C.c_void_p(a.data_ptr())
        return a.ctypes.data_as(C.c_void_p)
    res = ircur_result()
    _check(_lib().ircur_solve_host(ctx, hp(D_host), hp(L_host), hp(S_host), C.byref(res)),
           "ircur_solve_host")
    return res


def ircur_sample_indices(seed, draw, axis, n, m, out, stream=None):
    _check(_lib().ircur_sample_indices(seed, draw, axis, n, m, _ptr(out), stream), "ircur_sample_indices")


def ircur_get_cur(ctx, D, ldD, C=None, U=None, R=None):
    _check(_lib().ircur_get_cur(ctx, _ptr(D), ldD, _ptr(C), _ptr(U), _ptr(R)), "ircur_get_cur")


def ircur_set_trace(ctx, enable):
    _check(_lib().ircur_set_trace(ctx, int(bool(enable))), "ircur_set_trace")


def ircur_get_trace(ctx, max_iter):
    """Per-iteration kernel spans (us) of the last traced solve: list of
    (core Phase I, core SVD, panel pass, panel pass after its wait for the SVD)."""
    buf = (C.c_double * (4 * max_iter))()
    cnt = C.c_int32()
    _check(_lib().ircur_get_trace(ctx, buf, C.byref(cnt)), "ircur_get_trace")
    return [tuple(buf[4 * k + q] for q in range(4)) for k in range(cnt.value)]


def ircur_solve_noalloc(params: ircur_params, D, ldD, A, B, stream=None):
    """Allocation-free IRCUR-F solve (see include/ircur.h): writes the factors
    into the caller's device tensors A (n1 x r) and B (r x n2); L = A B."""
    res = ircur_result()
    _check(_lib().ircur_solve_noalloc(C.byref(params), _ptr(D), ldD, _ptr(A), _ptr(B), C.byref(res), stream),
           "ircur_solve_noalloc")
    return res


def ircur_get_svd(ctx, W, sigma, V):
    _check(_lib().ircur_get_svd(ctx, _ptr(W), _ptr(sigma), _ptr(V)), "ircur_get_svd")


def ircur_set_record(ctx, enable):
    _check(_lib().ircur_set_record(ctx, int(bool(enable))), "ircur_set_record")


def ircur_backward(ctx, D, ldD, dL, lddL, dS, lddS, dD, lddD):
    _check(_lib().ircur_backward(ctx, _ptr(D), ldD, _ptr(dL), lddL, _ptr(dS), lddS, _ptr(dD), lddD),
           "ircur_backward")


def ircur_batch_create(params_list, stream=None):
    n = len(params_list)
    arr = (ircur_params * n)(*params_list)
    b = C.c_void_p()
    _check(_lib().ircur_batch_create(arr, n, stream, C.byref(b)), "ircur_batch_create")
    return b


def ircur_batch_destroy(b):
    _lib().ircur_batch_destroy(b)


def ircur_batch_solve(b, Ds, lds):
    """Ds: device tensors (or raw pointers), lds: leading dimensions; returns the results."""
    n = len(Ds)
    ptrs = (C.c_void_p * n)(*[d.data_ptr() if hasattr(d, "data_ptr") else d for d in Ds])
    ldv = (C.c_int64 * n)(*lds)
    res = (ircur_result * n)()
    status = _lib().ircur_batch_solve(b, ptrs, ldv, res)
    return status, list(res)


def ircur_batch_instance(b, i):
    return C.c_void_p(_lib().ircur_batch_instance(b, i))


# ---------------------------------------------------------------- convenience layer
@dataclass
class Result:
    iters: int
    converged: bool
    flags: int
    svd_steps: int
    final_err: float
    zeta0: float
    zeta_next: float


class IRCUR:
    """One IRCUR problem shape bound to a CUDA device and stream.

    solver = IRCUR(n1, n2, r, resample=True)
    res = solver.solve(D)                 # D: float32 CUDA tensor, n1 x n2
    L, S = solver.reconstruct(D)          # dense outputs
    """

    def __init__(self, n1, n2, r, *, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=100,
                 resample=True, seed=0, precision=IRCUR_PRECISION_FP32, svd_form=0, stream=None):
        import torch
        self.p = ircur_params(n1=n1, n2=n2, r=r, nI=nI, nJ=nJ, zeta0=zeta0, gamma=gamma, tol=tol,
                              max_iter=max_iter, resample=int(bool(resample)), seed=seed,
                              precision=precision, svd_form=svd_form)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = ircur_create(self.p, C.c_void_p(self.stream.cuda_stream))
        self.nI = nI if nI else sample_size(4, r, n1)
        self.nJ = nJ if nJ else sample_size(4, r, n2)
        self.last = None
        self.solves = 0  # solves issued through this handle (ircur_unrolled checks it)

    @classmethod
    def _view(cls, ctx, p, stream, owner):
        """A non-owning handle on a context that `owner` (a batch) holds."""
        self = cls.__new__(cls)
        self.p, self.stream, self._ctx, self._owner = p, stream, ctx, owner
        self.nI = p.nI if p.nI else sample_size(4, p.r, p.n1)
        self.nJ = p.nJ if p.nJ else sample_size(4, p.r, p.n2)
        self.last = None
        self.solves = 0
        return self

    def close(self):
        if getattr(self, "_owner", None) is not None:
            self._ctx = None
            return
        if self._ctx:
            ircur_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, D, idx_I=None, idx_J=None):
        assert D.is_cuda and D.dtype.itemsize == 4 and D.stride(1) == 1
        self.solves += 1
        r = ircur_solve(self._ctx, D, D.stride(0), idx_I, idx_J)
        self.last = Result(r.iters, bool(r.converged), r.flags, r.svd_steps, r.final_err, r.zeta0,
                           r.zeta_next)
        return self.last

    def factors(self):
        import torch
        A = torch.empty((self.p.n1, self.p.r), dtype=torch.float32, device="cuda")
        B = torch.empty((self.p.r, self.p.n2), dtype=torch.float32, device="cuda")
        ircur_get_factors(self._ctx, A, B)
        return A, B

    def indices(self):
        import torch
        I = torch.empty(self.nI, dtype=torch.int32, device="cuda")
        J = torch.empty(self.nJ, dtype=torch.int32, device="cuda")
        sig = torch.empty(self.p.r, dtype=torch.float32, device="cuda")
        ircur_get_indices(self._ctx, I, J, sig)
        return I, J, sig

    def cur(self, D):
        """C (n1 x |J|), U (|I| x |J|), R (|I| x n2) of the last iterate (Alg. 1 output)."""
        import torch
        C = torch.empty((self.p.n1, self.nJ), dtype=torch.float32, device="cuda")
        U = torch.empty((self.nI, self.nJ), dtype=torch.float32, device="cuda")
        R = torch.empty((self.nI, self.p.n2), dtype=torch.float32, device="cuda")
        ircur_get_cur(self._ctx, D, D.stride(0), C, U, R)
        return C, U, R

    def errors(self):
        return ircur_get_errors(self._ctx, self.p.max_iter)

    def svd(self):
        """Alg. 2: L = W diag(sigma) V^T of the last iterate (W: n1 x r, V: n2 x r)."""
        import torch
        r = self.p.r
        W = torch.empty((self.p.n1, r), dtype=torch.float32, device="cuda")
        V = torch.empty((self.p.n2, r), dtype=torch.float32, device="cuda")
        sig = torch.empty(r, dtype=torch.float32, device="cuda")
        ircur_get_svd(self._ctx, W, sig, V)
        return W, sig, V

    def autotune(self, D, reps=3):
        """Time the pass-kernel launch shapes on D and keep the fastest (see include/ircur.h)."""
        out = ircur_tune_result()
        _check(_lib().ircur_autotune(self._ctx, _ptr(D), D.stride(0), reps, C.byref(out)), "ircur_autotune")
        return out.as_dict()

    def record(self, enable=True):
        """Make the following solves record their iterations for backward (IRCUR-F)."""
        ircur_set_record(self._ctx, enable)

    def backward(self, D, dL=None, dS=None, dD=None):
        """dD = d<dL, L>/dD + d<dS, S>/dD for the last recorded solve (see include/ircur.h)."""
        import torch
        if dD is None:
            dD = torch.empty((self.p.n1, self.p.n2), dtype=torch.float32, device=D.device)
        for t in (dL, dS):
            assert t is None or (t.is_cuda and t.dtype == torch.float32 and t.stride(1) == 1)
        ircur_backward(self._ctx, D, D.stride(0), dL, dL.stride(0) if dL is not None else 0,
                       dS, dS.stride(0) if dS is not None else 0, dD, dD.stride(0))
        return dD

    def reconstruct(self, D=None, with_sparse=True, L=None, S=None):
        import torch
        n1, n2 = self.p.n1, self.p.n2
        if L is None:
            L = torch.empty((n1, n2), dtype=torch.float32, device="cuda")
        if with_sparse and S is None:
            S = torch.empty((n1, n2), dtype=torch.float32, device="cuda")
        if not with_sparse:
            S = None
        ircur_reconstruct(self._ctx, D, D.stride(0) if D is not None else 0, L, L.stride(0),
                          S, S.stride(0) if S is not None else 0)
        return L, S

    def stream_columns(self, Dnew, iters=0, with_sparse=True):
        """New columns (n1 x c, row-major, on the device) against the last
        solve's CUR model: returns (L, S) for them (S None without with_sparse)."""
        import torch
        assert Dnew.is_cuda and Dnew.dtype == torch.float32 and Dnew.stride(1) == 1
        n1, c = Dnew.shape
        assert n1 == self.p.n1
        L = torch.empty((n1, c), dtype=torch.float32, device="cuda")
        S = torch.empty((n1, c), dtype=torch.float32, device="cuda") if with_sparse else None
        ircur_stream_columns(self._ctx, Dnew, Dnew.stride(0), c, iters, L, L.stride(0),
                             S, S.stride(0) if S is not None else 0)
        return L, S


def _make_function():
    import torch

    class _Unrolled(torch.autograd.Function):
        """D -> (L, S) of a recording IRCUR-F solve; backward through ircur_backward."""

        @staticmethod
        def forward(ctx, D, solver):
            solver.solve(D)
            L, S = solver.reconstruct(D)
            ctx.solver = solver
            ctx.generation = solver.solves
            ctx.save_for_backward(D)
            return L, S

        @staticmethod
        def backward(ctx, dL, dS):
            if ctx.solver.solves != ctx.generation:
                # the solver's recording now belongs to a later solve
                raise IrcurError(IRCUR_ESTATE, "ircur_unrolled backward: the solver ran another solve "
                                                "after this forward")
            (D,) = ctx.saved_tensors
            dL = dL.contiguous() if dL is not None else None
            dS = dS.contiguous() if dS is not None else None
            return ctx.solver.backward(D, dL, dS), None

    return _Unrolled


_FUNCTION = None


def ircur_unrolled(D, solver):
    """Differentiable (L, S) = IRCUR-F(D) for a solver made with resample=False;
    the solver records its iterations and the backward pass runs the
    hand-written adjoint.  Gradients flow to D only."""
    global _FUNCTION
    if _FUNCTION is None:
        _FUNCTION = _make_function()
    if not getattr(solver, "_recording", False):
        solver.record(True)
        solver._recording = True
    return _FUNCTION.apply(D, solver)


class IRCURBatch:
    """Independent IRCUR problems solved together (one kernel launch per
    iteration step for the whole batch).

    batch = IRCURBatch([dict(n1=500, n2=400, r=3), dict(n1=900, n2=900, r=6, resample=False)])
    results = batch.solve([D0, D1])       # list of Result
    L1, S1 = batch[1].reconstruct(D1)     # every IRCUR getter, per instance
    """

    def __init__(self, problems, stream=None):
        import torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = []
        for q in problems:
            q = dict(q)
            self.params.append(ircur_params(
                n1=q["n1"], n2=q["n2"], r=q["r"], nI=q.get("nI", 0), nJ=q.get("nJ", 0),
                zeta0=q.get("zeta0", 0.0), gamma=q.get("gamma", 0.7), tol=q.get("tol", 1e-5),
                max_iter=q.get("max_iter", 100), resample=int(bool(q.get("resample", True))),
                seed=q.get("seed", 0), precision=0, svd_form=q.get("svd_form", 0)))
        self._b = ircur_batch_create(self.params, C.c_void_p(self.stream.cuda_stream))
        self._views = [IRCUR._view(ircur_batch_instance(self._b, i), p, self.stream, self)
                       for i, p in enumerate(self.params)]
        self.last = None

    def __len__(self):
        return len(self.params)

    def __getitem__(self, i):
        return self._views[i]

    def solve(self, Ds):
        assert len(Ds) == len(self.params)
        for D in Ds:
            assert D.is_cuda and D.dtype.itemsize == 4 and D.stride(1) == 1
        status, res = ircur_batch_solve(self._b, Ds, [D.stride(0) for D in Ds])
        self.last = [Result(r.iters, bool(r.converged), r.flags, r.svd_steps, r.final_err, r.zeta0,
                            r.zeta_next) for r in res]
        for v, r in zip(self._views, self.last):
            v.last = r
        _check(status, "ircur_batch_solve")
        return self.last

    def autotune(self, Ds, reps=3):
        """Time the batched pass-kernel launch shapes on Ds and keep the fastest."""
        n = len(Ds)
        ptrs = (C.c_void_p * n)(*[d.data_ptr() for d in Ds])
        ldv = (C.c_int64 * n)(*[d.stride(0) for d in Ds])
        out = ircur_tune_result()
        _check(_lib().ircur_batch_autotune(self._b, ptrs, ldv, reps, C.byref(out)), "ircur_batch_autotune")
        return out.as_dict()

    def close(self):
        if self._b:
            for v in self._views:
                v._ctx = None
            ircur_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sample_indices(seed, draw, axis, n, m):
    """Device sampler (one draw): sorted uniform m-subset of [0, n)."""
    import torch
    out = torch.empty(m, dtype=torch.int32, device="cuda")
    ircur_sample_indices(seed, draw, axis, n, m, out, _stream_handle())
    return out
