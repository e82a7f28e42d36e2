"""Plain FP64 CPU oracle for IRCUR (Iterated Robust CUR), Cai, Hamm, Huang, Li,
Wang, "Rapid Robust Principal Component Analysis: CUR Accelerated Inexact Low
Rank Estimation" (arXiv 2010.07422).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library and imports
nothing but numpy.

Every function follows the paper's steps in the paper's order and notation:

* ``hard_threshold``   -- the operator T_zeta of Sec. 3.2 (strict ``>``).
* ``truncated_svd``    -- H_r, the best rank-r approximation of Sec. 3.1, taken
                          from a full LAPACK SVD (a library primitive).
* ``pinv_from_svd``    -- Moore-Penrose inverse of H_r(U), Thm 1 / Sec. 3.1.
* ``cur_product``      -- C U^+ R, Thm 1.
* ``sample_indices``   -- uniform sampling of I, J (Alg. 1, Thm 2) with a
                          counter-based splitmix64 stream (see its docstring).
* ``ircur``            -- Algorithm 1 (Phase I, Phase II, stopping criterion
                          of Sec. 3.3), IRCUR-F and IRCUR-R (Sec. 3.4).
* ``dense_outputs``    -- L = C U^+ R written out in full, and the sparse part
                          S = T_zeta(D - L) at the threshold the next Phase I
                          would use.
* ``cur_to_svd``       -- Algorithm 2 (CUR to SVD conversion).
* ``stream_columns``   -- new columns through Alg. 1 with the final iterate's
                          column space C U^+ held fixed (an extension the
                          paper leaves implicit: IRCUR-F touches only the
                          rows I of a column, Sec. 3.4).

Readings taken where the paper is silent:
* ``log`` in |I| = c r log n is the natural log; |I| is rounded up.
* zeta_{k+1} = gamma^k zeta_0 (Alg. 1): the first iteration (k = 0) thresholds
  at zeta_0 itself.  gamma^k is formed by repeated FP64 multiplication.
* Alg. 1 assigns [S]_{:,J} and then [S]_{I,:}; the (I,J) block therefore holds
  the value of the second assignment (the row panel).
* IRCUR-R uses draw k of the index stream at iteration k (draw 0 at k = 0);
  IRCUR-F uses draw 0 throughout.  e_{k+1} is measured on the index sets that
  built iterate k+1.
* The pseudo-inverse treats singular values <= max(|I|,|J|) * eps * sigma_1 as
  zero, so a rank-deficient core uses its numerical rank.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# Sec. 3.2: hard-thresholding operator
# --------------------------------------------------------------------------


def hard_threshold(X, zeta):
    """[T_zeta X]_ij = X_ij if |X_ij| > zeta, else 0 (Sec. 3.2, strict >)."""
    X = np.asarray(X, dtype=np.float64)
    return np.where(np.abs(X) > zeta, X, 0.0)


# --------------------------------------------------------------------------
# Sec. 3.1 / Thm 1: rank-r truncation, pseudo-inverse, CUR product
# --------------------------------------------------------------------------


def truncated_svd(U, r):
    """H_r(U) = W_r Sigma_r V_r^T, the best rank-r approximation (Sec. 3.1).

    Returns (W_r, s_r, V_r) with W_r: |I| x r, s_r: r, V_r: |J| x r.
    The full SVD comes from LAPACK (numpy.linalg.svd), used as a primitive.
    """
    U = np.asarray(U, dtype=np.float64)
    W, s, Vt = np.linalg.svd(U, full_matrices=False)
    r = min(r, s.shape[0])
    return W[:, :r], s[:r], Vt[:r, :].T


def numerical_rank(s, shape):
    """Number of singular values above max(shape) * eps * s_1."""
    if s.size == 0 or s[0] == 0.0:
        return 0
    tol = max(shape) * np.finfo(np.float64).eps * s[0]
    return int(np.sum(s > tol))


def pinv_from_svd(W_r, s_r, V_r, shape):
    """Moore-Penrose inverse of H_r(U) = W_r diag(s_r) V_r^T (Thm 1).

    (W diag(s) V^T)^+ = V diag(1/s) W^T over the numerically nonzero s.
    Returns (U_pinv, rank) with U_pinv of shape |J| x |I|.
    """
    k = numerical_rank(s_r, shape)
    return (V_r[:, :k] / s_r[:k]) @ W_r[:, :k].T, k


def cur_product(C, U_pinv, R):
    """C U^+ R (Thm 1): the CUR reconstruction of a matrix."""
    return np.asarray(C, np.float64) @ np.asarray(U_pinv, np.float64) @ np.asarray(R, np.float64)


# --------------------------------------------------------------------------
# Alg. 1 / Thm 2: uniform sampling of I and J with a counter-based stream
# --------------------------------------------------------------------------

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """splitmix64 output for state x (Steele, Lea, Flood, OOPSLA 2014):
    z = x + 0x9e3779b97f4a7c15; z = (z ^ z>>30) * 0xbf58476d1ce4e5b9;
    z = (z ^ z>>27) * 0x94d049bb133111eb; return z ^ z>>31 (all mod 2^64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def sample_size(c, r, n):
    """|I| = ceil(c * r * ln n), capped at n (Sec. 3.5, natural log, rounded up)."""
    return int(min(n, math.ceil(c * r * math.log(n))))


def sample_indices(seed, draw, axis, n, m):
    """Uniform m-subset of [0, n) for draw `draw` on `axis` (0 = rows, 1 = cols).

    Every element i gets the key splitmix64(splitmix64(splitmix64(seed) ^
    (2*draw + axis)) ^ i); the m elements with the smallest keys (ties broken
    by the smaller index) form the sample, returned in ascending order.  The
    keys are i.i.d. uniform, so every m-subset is equally likely: this is
    uniform sampling without replacement (Alg. 1; Thm 2 states the bound for
    sampling with replacement, and distinct indices only help the rank).
    """
    if not (0 < m <= n):
        raise ValueError("need 0 < m <= n")
    s = splitmix64(np.uint64(seed))
    s = splitmix64(s ^ np.uint64(2 * draw + axis))
    keys = splitmix64(s ^ np.arange(n, dtype=np.uint64))
    order = np.lexsort((np.arange(n), keys))  # primary key: keys, then index
    return np.sort(order[:m]).astype(np.int64)


# --------------------------------------------------------------------------
# Alg. 1: IRCUR
# --------------------------------------------------------------------------


@dataclass
class IrcurResult:
    C: np.ndarray  # n1 x |J|   [D - S]_{:,J} of the last iteration
    U: np.ndarray  # |I| x |J|  H_r([D - S]_{I,J})
    U_pinv: np.ndarray  # |J| x |I|
    R: np.ndarray  # |I| x n2   [D - S]_{I,:}
    I: np.ndarray
    J: np.ndarray
    W_r: np.ndarray
    s_r: np.ndarray
    V_r: np.ndarray
    iters: int
    converged: bool
    errs: list = field(default_factory=list)  # e_1, e_2, ... (Sec. 3.3)
    zetas: list = field(default_factory=list)  # zeta used at each iteration
    zeta_next: float = 0.0  # gamma^K zeta_0, the next Phase I threshold
    ranks: list = field(default_factory=list)
    history: list = field(default_factory=list)  # optional per-iteration snapshots


def ircur(D, r, zeta0, gamma, tol, max_iter, *, nI=None, nJ=None, c=4.0,
          resample=False, seed=0, index_draws=None, keep_history=False):
    """Algorithm 1 (IRCUR), FP64, on the panels only.

    D            : n1 x n2 array (promoted to FP64).
    zeta0 <= 0   : use max|D| (with strict >, the first Phase I then keeps S = 0).
    index_draws  : optional callable draw -> (I, J); otherwise `sample_indices`.
    resample     : False = IRCUR-F (draw 0 throughout), True = IRCUR-R.
    Returns an IrcurResult holding the CUR factors of the final iterate.
    """
    D = np.asarray(D, dtype=np.float64)
    n1, n2 = D.shape
    if nI is None:
        nI = sample_size(c, r, n1)
    if nJ is None:
        nJ = sample_size(c, r, n2)
    if zeta0 is None or zeta0 <= 0:
        zeta0 = float(np.max(np.abs(D)))

    def draw(k):
        if index_draws is not None:
            I, J = index_draws(k)
            return np.asarray(I, np.int64), np.asarray(J, np.int64)
        return sample_indices(seed, k, 0, n1, nI), sample_indices(seed, k, 1, n2, nJ)

    # L_0 = 0, S_0 = 0, k = 0; e_0 = 1 so the loop body runs at least once.
    C_k = U_pinv_k = R_k = None
    res = None
    zeta = float(zeta0)
    errs, zetas, ranks, history = [], [], [], []
    I, J = draw(0)
    k = 0
    e = 1.0
    while e > tol and k < max_iter:
        if resample:
            I, J = draw(k)
        # ---- Phase I: zeta_{k+1} = gamma^k zeta_0, threshold the panels of D - L_k
        zetas.append(zeta)
        D_rows = D[I, :]  # D_{I,:}
        D_cols = D[:, J]  # D_{:,J}
        if C_k is None:  # L_0 = 0
            L_rows = np.zeros_like(D_rows)
            L_cols = np.zeros_like(D_cols)
        else:  # [L_k]_{I,:} = [C_k]_{I,:} U_k^+ R_k ; [L_k]_{:,J} = C_k U_k^+ [R_k]_{:,J}
            L_rows = C_k[I, :] @ U_pinv_k @ R_k
            L_cols = C_k @ U_pinv_k @ R_k[:, J]
        S_cols = hard_threshold(D_cols - L_cols, zeta)  # [S_{k+1}]_{:,J}
        S_rows = hard_threshold(D_rows - L_rows, zeta)  # [S_{k+1}]_{I,:}
        S_cols[I, :] = S_rows[:, J]  # the second assignment owns the (I,J) block
        # ---- Phase II: C, U = H_r(core), R  (L_{k+1} = C U^+ R is not formed)
        C_new = D_cols - S_cols
        R_new = D_rows - S_rows
        core = R_new[:, J]  # [D - S_{k+1}]_{I,J}
        W_r, s_r, V_r = truncated_svd(core, r)
        U_new = (W_r * s_r) @ V_r.T
        U_pinv_new, rank = pinv_from_svd(W_r, s_r, V_r, core.shape)
        # ---- stopping criterion (Sec. 3.3) on the sets that built iterate k+1
        L_rows_new = C_new[I, :] @ U_pinv_new @ R_new
        L_cols_new = C_new @ U_pinv_new @ R_new[:, J]
        num = (np.linalg.norm(R_new - L_rows_new) + np.linalg.norm(C_new - L_cols_new))
        den = np.linalg.norm(D_rows) + np.linalg.norm(D_cols)
        e = num / den if den > 0 else 0.0
        errs.append(e)
        ranks.append(rank)
        if keep_history:
            history.append(dict(I=I.copy(), J=J.copy(), zeta=zeta, C=C_new, R=R_new,
                                core=core, U_pinv=U_pinv_new, S_rows=S_rows, S_cols=S_cols,
                                W_r=W_r, s_r=s_r, V_r=V_r))
        C_k, U_pinv_k, R_k = C_new, U_pinv_new, R_new
        res = (U_new, W_r, s_r, V_r)
        zeta = zeta * gamma
        k += 1

    U_new, W_r, s_r, V_r = res
    return IrcurResult(C=C_k, U=U_new, U_pinv=U_pinv_k, R=R_k, I=I, J=J, W_r=W_r, s_r=s_r,
                       V_r=V_r, iters=k, converged=bool(e <= tol), errs=errs, zetas=zetas,
                       zeta_next=zeta, ranks=ranks, history=history)


def dense_outputs(D, result, with_sparse=True):
    """L = C U^+ R in full and S = T_{zeta_next}(D - L) (zeta_next = gamma^K zeta_0)."""
    L = cur_product(result.C, result.U_pinv, result.R)
    if not with_sparse:
        return L, None
    return L, hard_threshold(np.asarray(D, np.float64) - L, result.zeta_next)


def entries(result, rows, cols):
    """L_ij = C_{i,:} U^+ R_{:,j} at the listed (i, j) pairs, one by one."""
    rows = np.asarray(rows, np.int64)
    cols = np.asarray(cols, np.int64)
    left = result.C[rows, :] @ result.U_pinv  # one row of C U^+ per sample
    return np.einsum("kt,tk->k", left, result.R[:, cols])


# --------------------------------------------------------------------------
# Algorithm 2: CUR to SVD
# --------------------------------------------------------------------------


def cur_to_svd(C, U_pinv, R):
    """Algorithm 2: [Q_C, R_C] = qr(C); [Q_R, R_R] = qr(R^T);
    [W_U, Sigma, V_U] = svd(R_C U^+ R_R^T); W = Q_C W_U; V = Q_R V_U."""
    Q_C, R_C = np.linalg.qr(np.asarray(C, np.float64))
    Q_R, R_R = np.linalg.qr(np.asarray(R, np.float64).T)
    W_U, sigma, V_Ut = np.linalg.svd(R_C @ U_pinv @ R_R.T)
    return Q_C @ W_U, sigma, Q_R @ V_Ut.T


# --------------------------------------------------------------------------
# Streaming extension: new columns against a fixed CUR model
# --------------------------------------------------------------------------


def stream_columns(Dnew, result, zeta0, gamma, iters):
    """New columns d (the columns of Dnew, n1 x c) go through Alg. 1 with the
    final iterate's C and U^+ (and its row set I) held fixed.  The paper does
    not state this step; it follows from Alg. 1 because a column enters the
    iteration only through its entries on the rows I (R = D_{I,:} - S_{I,:}),
    and L = C U^+ R then extends it to all rows.  Per column, from L_0 = 0:

        for t = 0 .. iters-1:   zeta_t = gamma^t zeta_0
            S_I = T_{zeta_t}(d_I - [L_t]_I)          (Phase I, on the rows I)
            r   = d_I - S_I                           (the column's entry of R)
            [L_{t+1}]_I = C_{I,:} U^+ r               (Phase II, C and U^+ fixed)
        L = C U^+ r,  S = T_{zeta_iters}(d - L)      (as ``dense_outputs``)

    Returns (L, S), both n1 x c, FP64."""
    Dnew = np.asarray(Dnew, dtype=np.float64)
    if Dnew.ndim == 1:
        Dnew = Dnew[:, None]
    C, U_pinv, I = result.C, result.U_pinv, result.I
    d_I = Dnew[I, :]
    L_I = np.zeros_like(d_I)
    zeta = float(zeta0)
    r = d_I
    for _ in range(iters):
        S_I = hard_threshold(d_I - L_I, zeta)
        r = d_I - S_I
        L_I = C[I, :] @ (U_pinv @ r)
        zeta = zeta * gamma
    L = C @ (U_pinv @ r)
    return L, hard_threshold(Dnew - L, zeta)
