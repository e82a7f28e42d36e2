"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact
threshold values at hand-built ties (Sec. 3.2), Thm 1 by brute force over all
index sets of tiny matrices, the Penrose conditions, Eckart-Young through a
different LAPACK routine (symmetric eigenvalues), the pure low-rank closed form,
the projection form of the stopping criterion, L(I,J) = U, planted recovery at
the paper's success threshold (Sec. 4.1.1), equivariances, a dense restatement
of Alg. 1 on tiny inputs, the published splitmix64 outputs and the sampler's
inclusion probabilities.
"""

import itertools
import math
import os

import numpy as np
import pytest

from oracle import (cur_product, cur_to_svd, dense_outputs, entries, hard_threshold, ircur,
                    numerical_rank, pinv_from_svd, sample_indices, sample_size, splitmix64,
                    truncated_svd)
from paper_2010_07422_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Sec. 3.2
def test_hard_threshold_exact_values_and_ties():
    zeta = 0.75
    X = np.array([[0.75, -0.75, 0.7500000000000001, -0.7500000000000001],
                  [0.0, 3.0, -2.5, 0.74999999999999989]])
    want = np.array([[0.0, 0.0, 0.7500000000000001, -0.7500000000000001],
                     [0.0, 3.0, -2.5, 0.0]])
    got = hard_threshold(X, zeta)
    assert np.array_equal(got, want)
    # the kept entries are the inputs bit for bit
    assert got[0, 2] == X[0, 2] and got[1, 2] == X[1, 2]


# ---------------------------------------------------------------- Thm 1
def _subsets(n, kmin):
    for k in range(kmin, n + 1):
        yield from itertools.combinations(range(n), k)


def _exact_rank(M):
    """Rank of an integer matrix by fraction-free (Bareiss) elimination in Python
    integers: exact, and independent of LAPACK and of any tolerance."""
    A = [[int(v) for v in row] for row in np.asarray(M)]
    rows, cols = len(A), len(A[0]) if A else 0
    rank, prev = 0, 1
    for c in range(cols):
        piv = next((i for i in range(rank, rows) if A[i][c] != 0), None)
        if piv is None:
            continue
        A[rank], A[piv] = A[piv], A[rank]
        for i in range(rank + 1, rows):
            for j in range(c + 1, cols):
                A[i][j] = (A[i][j] * A[rank][c] - A[i][c] * A[rank][j]) // prev
            A[i][c] = 0
        prev = A[rank][c]
        rank += 1
    return rank


def test_exact_rank_helper():
    assert _exact_rank(np.eye(4)) == 4
    assert _exact_rank([[1, 2, 3], [2, 4, 6], [1, 0, 1]]) == 2
    assert _exact_rank(np.zeros((3, 2))) == 0
    assert _exact_rank([[0, 0, 5], [0, 0, 1]]) == 1
    rng = np.random.default_rng(1)
    W, V = rng.integers(-3, 4, (7, 3)), rng.integers(-3, 4, (5, 3))
    assert _exact_rank(W @ V.T) == min(_exact_rank(W), _exact_rank(V), 3)


@pytest.mark.parametrize("r", [1, 2, 3])
def test_cur_identity_bruteforce(r):
    """L = C U^+ R for every I, J with rank(U) = rank(L) (Thm 1), all subsets.

    The rank of each core comes from exact integer elimination, not from the
    oracle's tolerance: where the core is rank deficient the oracle's
    pseudo-inverse must use exactly that smaller rank (Sec. 3.1 truncation of a
    matrix whose trailing singular values are zero)."""
    rng = np.random.default_rng(100 + r)
    n = 6
    W = rng.integers(-3, 4, size=(n, r)).astype(float)
    V = rng.integers(-3, 4, size=(n, r)).astype(float)
    W[1] = W[0]  # repeated rows/cols make some samples rank deficient
    V[2] = 0.0
    L = W @ V.T
    assert _exact_rank(L) == r
    holds = fails_deficient = deficient = 0
    for I in _subsets(n, r):
        for J in _subsets(n, r):
            C, U, R = L[:, J], L[np.ix_(I, J)], L[I, :]
            W_r, s_r, V_r = truncated_svd(U, r)
            Up, rank = pinv_from_svd(W_r, s_r, V_r, U.shape)
            err = np.linalg.norm(cur_product(C, Up, R) - L)
            true_rank = _exact_rank(U)
            assert rank == true_rank, (I, J, rank, true_rank)
            if true_rank == r:
                assert err <= 1e-10 * np.linalg.norm(L)
                holds += 1
            else:
                deficient += 1
                if err > 1e-8 * np.linalg.norm(L):
                    fails_deficient += 1
    assert holds > 100
    assert deficient > 0
    assert fails_deficient > 0  # rank(U) < rank(L): the identity need not hold


def test_numerical_rank_cutoff_is_strict_and_fp64():
    """The pseudo-inverse drops singular values s <= max(|I|,|J|) * eps64 * s_1:
    at the cutoff itself the value is dropped (strict >), just above it kept, and
    a value far below FP32 resolution but above the FP64 cutoff is kept."""
    eps = np.finfo(np.float64).eps
    for shape in [(2, 2), (7, 3), (185, 185)]:
        tol = max(shape) * eps
        assert numerical_rank(np.array([1.0, tol]), shape) == 1
        assert numerical_rank(np.array([1.0, 2.0 * tol]), shape) == 2
        assert numerical_rank(np.array([4.0, 4.0 * tol]), shape) == 1
        assert numerical_rank(np.array([1.0, 1e-10]), shape) == 2
        assert numerical_rank(np.array([1.0, 0.5, 0.0]), shape) == 2
    assert numerical_rank(np.array([0.0, 0.0]), (3, 3)) == 0
    assert numerical_rank(np.array([]), (3, 3)) == 0
    # through the SVD: a diagonal core with an exactly known spectrum
    U = np.diag([3.0, 1.0, 3.0 * 2 * eps, 0.0])
    W_r, s_r, V_r = truncated_svd(U, 4)
    Up, rank = pinv_from_svd(W_r, s_r, V_r, U.shape)
    assert rank == 2
    assert np.array_equal(np.abs(Up), np.diag([1 / 3.0, 1.0, 0.0, 0.0]))


# ---------------------------------------------------------------- pinv, H_r
def test_pinv_penrose_conditions():
    rng = np.random.default_rng(7)
    for (m, n, r) in [(9, 7, 3), (12, 12, 5), (5, 8, 2)]:
        Uc = rng.standard_normal((m, n))
        W_r, s_r, V_r = truncated_svd(Uc, r)
        A = (W_r * s_r) @ V_r.T
        X, rank = pinv_from_svd(W_r, s_r, V_r, Uc.shape)
        assert rank == r and X.shape == (n, m)
        tol = 1e-12 * max(1.0, np.linalg.norm(A)) * max(1.0, np.linalg.norm(X))
        assert np.linalg.norm(A @ X @ A - A) <= tol
        assert np.linalg.norm(X @ A @ X - X) <= tol
        assert np.linalg.norm((A @ X).T - A @ X) <= tol
        assert np.linalg.norm((X @ A).T - X @ A) <= tol


def test_truncated_svd_eckart_young():
    """||U - H_r(U)||_F^2 equals the sum of the m - r smallest eigenvalues of U^T U."""
    rng = np.random.default_rng(8)
    for (m, r) in [(10, 3), (20, 5), (15, 1)]:
        U = rng.standard_normal((m, m))
        W_r, s_r, V_r = truncated_svd(U, r)
        H = (W_r * s_r) @ V_r.T
        lam = np.linalg.eigvalsh(U.T @ U)  # ascending, a different LAPACK driver
        assert abs(np.linalg.norm(U - H) ** 2 - lam[: m - r].sum()) <= 1e-10 * lam.sum()
        assert np.allclose(np.sort(s_r ** 2), lam[m - r:], rtol=1e-10)
        assert np.allclose(W_r.T @ W_r, np.eye(r), atol=1e-12)
        assert np.allclose(V_r.T @ V_r, np.eye(r), atol=1e-12)
        assert np.linalg.matrix_rank(H) == r


# ---------------------------------------------------------------- Alg. 1 special cases
def test_first_iteration_with_zeta0_maxD_thresholds_nothing():
    p = synth.planted(120, 90, 3, 0.1, seed=3)
    res = ircur(p.D, 3, 0, 0.7, 1e-5, 1, resample=True, seed=5, keep_history=True)
    h = res.history[0]
    assert h["zeta"] == float(np.max(np.abs(p.D.astype(np.float64))))
    assert not np.any(h["S_rows"]) and not np.any(h["S_cols"])
    D = p.D.astype(np.float64)
    assert np.array_equal(h["R"], D[h["I"], :]) and np.array_equal(h["C"], D[:, h["J"]])


@pytest.mark.parametrize("resample", [False, True])
def test_pure_lowrank_recovered_in_one_iteration(resample):
    """S = 0 and rank(D) = r: by Thm 1 the first iterate is D itself, e_1 ~ 0."""
    rng = np.random.default_rng(11)
    n1, n2, r = 150, 130, 4
    D = rng.standard_normal((n1, r)) @ rng.standard_normal((r, n2))
    res = ircur(D, r, 0, 0.7, 1e-10, 50, resample=resample, seed=2)
    assert res.iters == 1 and res.converged
    assert res.errs[0] <= 1e-13
    L, _ = dense_outputs(D, res, with_sparse=False)
    assert np.linalg.norm(L - D) <= 1e-12 * np.linalg.norm(D)


def test_stopping_criterion_projection_form_and_core_identity():
    """e_{k+1} computed literally equals the projection form
    ||(I - W_r W_r^T) R|| + ||C (I - V_r V_r^T)||, and L_{k+1}(I,J) = U."""
    p = synth.planted(300, 260, 4, 0.1, seed=4)
    res = ircur(p.D, 4, 0, 0.7, 1e-5, 12, resample=True, seed=9, keep_history=True)
    D = p.D.astype(np.float64)
    for k, h in enumerate(res.history):
        W, V = h["W_r"], h["V_r"]
        R, C = h["R"], h["C"]
        num = np.linalg.norm(R - W @ (W.T @ R)) + np.linalg.norm(C - (C @ V) @ V.T)
        den = np.linalg.norm(D[h["I"], :]) + np.linalg.norm(D[:, h["J"]])
        assert abs(num / den - res.errs[k]) <= 1e-10 * max(res.errs[k], 1e-300) + 1e-14
        # L_{k+1}(I,J) = C(I,:) U^+ R(:,J) = H_r(core)
        U = (W * h["s_r"]) @ V.T
        LIJ = C[h["I"], :] @ h["U_pinv"] @ R[:, h["J"]]
        assert np.linalg.norm(LIJ - U) <= 1e-10 * np.linalg.norm(U)
        # every entry of R_{k+1} and C_{k+1} is D_ij or the thresholded L_k
        assert np.all((R == D[h["I"], :]) | (h["S_rows"] != 0))


@pytest.mark.parametrize("resample", [False, True])
def test_planted_recovery_config0(resample):
    """n = 1000, r = 5, alpha = 0.1, |I| = |J| = ceil(4 r ln n) = 139, zeta_0 = max|D|,
    gamma = 0.7, tol = 1e-5: success per Sec. 4.1.1 (rel. error <= 1e-3)."""
    p = synth.planted(1000, 1000, 5, 0.1, seed=0)
    assert sample_size(4, 5, 1000) == 139
    res = ircur(p.D, 5, 0, 0.7, 1e-5, 100, resample=resample, seed=1)
    assert res.converged and res.iters < 60
    L, S = dense_outputs(p.D, res)
    Lt = p.L_true()
    err = np.linalg.norm(L - Lt) / np.linalg.norm(Lt)
    assert err <= 1e-3  # the paper's success criterion
    assert err <= 1e-4  # what tol = 1e-5 delivers in practice
    St = p.S_true()
    assert np.linalg.norm(S - St) / np.linalg.norm(St) <= 1e-4
    assert all(rk == 5 for rk in res.ranks)
    # the errors decay overall (linear convergence, Sec. 4.1.2)
    assert res.errs[-1] < 1e-3 * res.errs[0]


# ---------------------------------------------------------------- equivariances
def _fixed_draws(I, J):
    return lambda k: (I, J)


def test_scaling_by_power_of_two_is_exact():
    p = synth.planted(200, 180, 3, 0.1, seed=12)
    D = p.D.astype(np.float64)
    I = synth.random_subset(200, 40, 1)
    J = synth.random_subset(180, 40, 2)
    a = ircur(D, 3, 0, 0.7, 1e-6, 30, index_draws=_fixed_draws(I, J))
    b = ircur(D * 8.0, 3, 0, 0.7, 1e-6, 30, index_draws=_fixed_draws(I, J))
    assert a.iters == b.iters
    La, Sa = dense_outputs(D, a)
    Lb, Sb = dense_outputs(D * 8.0, b)
    assert np.linalg.norm(Lb - 8.0 * La) <= 1e-12 * np.linalg.norm(Lb)
    assert np.array_equal(Sb != 0, Sa != 0)


def test_transpose_equivariance():
    p = synth.planted(160, 200, 3, 0.1, seed=13)
    D = p.D.astype(np.float64)
    I = synth.random_subset(160, 40, 3)
    J = synth.random_subset(200, 45, 4)
    a = ircur(D, 3, 0, 0.7, 1e-7, 40, index_draws=_fixed_draws(I, J))
    b = ircur(D.T, 3, 0, 0.7, 1e-7, 40, index_draws=_fixed_draws(J, I))
    La, _ = dense_outputs(D, a, with_sparse=False)
    Lb, _ = dense_outputs(D.T, b, with_sparse=False)
    assert np.linalg.norm(Lb.T - La) <= 1e-9 * np.linalg.norm(La)


def test_index_order_does_not_matter():
    p = synth.planted(150, 150, 3, 0.1, seed=14)
    I = synth.random_subset(150, 36, 5)
    J = synth.random_subset(150, 36, 6)
    rng = np.random.default_rng(0)
    Ip, Jp = rng.permutation(I), rng.permutation(J)
    a = ircur(p.D, 3, 0, 0.7, 1e-7, 40, index_draws=_fixed_draws(I, J))
    b = ircur(p.D, 3, 0, 0.7, 1e-7, 40, index_draws=_fixed_draws(Ip, Jp))
    La, _ = dense_outputs(p.D, a, with_sparse=False)
    Lb, _ = dense_outputs(p.D, b, with_sparse=False)
    assert np.linalg.norm(Lb - La) <= 1e-9 * np.linalg.norm(La)


# ---------------------------------------------------------------- dense brute force
def _dense_ircur(D, r, zeta0, gamma, iters, I, J):
    """Alg. 1 with every matrix formed in full (tiny n only): L_k = C U^+ R as an
    n1 x n2 matrix, S_{k+1} thresholded everywhere, panels read off afterwards."""
    n1, n2 = D.shape
    L = np.zeros_like(D)
    zeta = zeta0
    for _ in range(iters):
        S = np.zeros_like(D)
        for i in range(n1):
            for j in range(n2):
                x = D[i, j] - L[i, j]
                if (j in J or i in I) and abs(x) > zeta:
                    S[i, j] = x
        C = (D - S)[:, J]
        R = (D - S)[I, :]
        Wf, sf, Vtf = np.linalg.svd((D - S)[np.ix_(I, J)])
        Up = Vtf[:r].T @ np.diag(1.0 / sf[:r]) @ Wf[:, :r].T
        L = C @ Up @ R
        zeta *= gamma
    return L


def test_dense_restatement_matches_panels():
    p = synth.planted(24, 20, 2, 0.1, seed=15)
    D = p.D.astype(np.float64)
    I = np.array([1, 4, 7, 9, 13, 18, 22])
    J = np.array([0, 3, 5, 8, 11, 16])
    for iters in (1, 2, 5):
        a = ircur(D, 2, 0, 0.7, 0.0, iters, index_draws=_fixed_draws(I, J))
        La, _ = dense_outputs(D, a, with_sparse=False)
        Lb = _dense_ircur(D, 2, float(np.abs(D).max()), 0.7, iters, list(I), list(J))
        assert np.linalg.norm(La - Lb) <= 1e-10 * np.linalg.norm(Lb)
    rows = np.array([0, 5, 23, 7])
    cols = np.array([19, 0, 4, 8])
    assert np.allclose(entries(a, rows, cols), La[rows, cols], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- Alg. 2
def test_cur_to_svd():
    p = synth.planted(200, 150, 4, 0.1, seed=16)
    res = ircur(p.D, 4, 0, 0.7, 1e-6, 60, seed=3)
    W, sig, V = cur_to_svd(res.C, res.U_pinv, res.R)
    L = cur_product(res.C, res.U_pinv, res.R)
    r = 4
    assert np.linalg.norm((W[:, :r] * sig[:r]) @ V[:, :r].T - L) <= 1e-10 * np.linalg.norm(L)
    assert np.allclose(W[:, :r].T @ W[:, :r], np.eye(r), atol=1e-12)
    assert np.allclose(V[:, :r].T @ V[:, :r], np.eye(r), atol=1e-12)


# ---------------------------------------------------------------- sampler
def test_splitmix64_published_outputs():
    vals = [int(line, 16) for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if line.strip() and not line.startswith("#")]
    golden = 0x9E3779B97F4A7C15
    for i, v in enumerate(vals):
        assert int(splitmix64(np.uint64((i * golden) % 2 ** 64))) == v


def test_sampler_sorted_distinct_and_uniform():
    n, m, draws = 20, 5, 4000
    counts = np.zeros(n)
    pair = 0
    for d in range(draws):
        s = sample_indices(77, d, d % 2, n, m)
        assert s.size == m and np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < n
        counts[s] += 1
        pair += (0 in s) and (1 in s)
    # inclusion probability m/n; chi-square with 19 dof, 0.999 quantile ~ 43.8
    expect = draws * m / n
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 43.8
    # pairwise inclusion probability m(m-1)/(n(n-1)) = 1/19
    p2 = m * (m - 1) / (n * (n - 1))
    assert abs(pair / draws - p2) < 4 * math.sqrt(p2 * (1 - p2) / draws)
    # edge cases: m = n returns everything, m = 1 works
    assert np.array_equal(sample_indices(1, 0, 0, 7, 7), np.arange(7))
    assert sample_indices(1, 0, 0, 7, 1).size == 1
    # draws and axes are independent streams
    assert not np.array_equal(sample_indices(1, 0, 0, 1000, 50), sample_indices(1, 0, 1, 1000, 50))
    assert not np.array_equal(sample_indices(1, 0, 0, 1000, 50), sample_indices(1, 1, 0, 1000, 50))


def test_sample_size_rule():
    assert sample_size(4, 5, 10000) == 185
    assert sample_size(4, 10, 4096) == 333
    assert sample_size(4, 2, 19200) == 79 and sample_size(4, 2, 3055) == 65
    assert sample_size(4, 10, 64) == 64  # capped at n
