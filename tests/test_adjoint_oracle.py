"""Pins of the FP64 adjoint oracle (oracle/ircur_adjoint.py) against what the
mathematics fixes, independently of the oracle's own code path:

* its forward equals Algorithm 1 as the main oracle runs it (IRCUR-F, the same
  index sets, exactly T iterations);
* its gradient equals central finite differences of the forward (FP64,
  h = 1e-6) along random directions, on a tiny instance whose threshold masks
  do not change within the step;
* the gradient of <dL, L_T> is supported on rows I and columns J only (the
  map reads D nowhere else), and the S-output adds exactly mask(S) * dS
  elsewhere;
* with no outliers flagged (zeta_0 above every residual) and T = 1, the map is
  L = D(:,J) H_r(D(I,J))^+ D(I,:), whose derivative along a direction that
  touches only D(:, j) for one j outside J is the CUR formula applied to that
  column: L(:, j) changes by C U^+ dD(I, j).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import ircur_adjoint as adj  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402


def _case(n1=64, n2=56, r=3, mI=20, mJ=18, alpha=0.1, seed=3):
    p = synth.planted(n1, n2, r, alpha, seed=seed)
    D = p.D.astype(np.float64)
    I = oracle.sample_indices(seed, 0, 0, n1, mI)
    J = oracle.sample_indices(seed, 0, 1, n2, mJ)
    return D, I, J


def test_forward_equals_algorithm_1():
    D, I, J = _case()
    T, z0, g = 6, None, 0.7
    z0 = float(np.abs(D).max())
    ref = oracle.ircur(D, 3, z0, g, 1e-300, T, nI=len(I), nJ=len(J), index_draws=lambda k: (I, J))
    assert ref.iters == T
    Lo, So = oracle.dense_outputs(D, ref)
    L, S = adj.unrolled_outputs(D, I, J, 3, z0, g, T)
    assert np.abs(L - Lo).max() <= 1e-10 * np.abs(Lo).max()
    assert np.abs(S - So).max() <= 1e-10 * np.abs(So).max()


@pytest.mark.parametrize("T,seed", [(1, 3), (5, 4), (12, 5)])
def test_gradient_matches_central_differences(T, seed):
    D, I, J = _case(seed=seed)
    # zeta_0 just above max|D| (at exactly max|D| the largest entry sits on the
    # threshold and any step moves it across)
    z0, g, h = 1.01 * float(np.abs(D).max()), 0.7, 1e-6
    rng = np.random.default_rng(seed)
    dL = rng.standard_normal(D.shape)
    dS = rng.standard_normal(D.shape)
    G = adj.unrolled_vjp(D, I, J, 3, z0, g, T, dL, dS)
    checked = 0
    for _ in range(6):
        V = rng.standard_normal(D.shape)
        mp = adj.masks(D + h * V, I, J, 3, z0, g, T)
        mm = adj.masks(D - h * V, I, J, 3, z0, g, T)
        if not all(np.array_equal(a, b) for a, b in zip(mp, mm)):
            continue  # the step crosses a threshold: not one smooth piece
        Lp, Sp = adj.unrolled_outputs(D + h * V, I, J, 3, z0, g, T)
        Lm, Sm = adj.unrolled_outputs(D - h * V, I, J, 3, z0, g, T)
        fd = (((Lp - Lm) * dL).sum() + ((Sp - Sm) * dS).sum()) / (2 * h)
        an = (G * V).sum()
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (fd, an)
        checked += 1
    assert checked >= 3


def test_gradient_support_rows_I_cols_J():
    D, I, J = _case(seed=6)
    z0 = float(np.abs(D).max())
    rng = np.random.default_rng(1)
    dL = rng.standard_normal(D.shape)
    G = adj.unrolled_vjp(D, I, J, 3, z0, 0.7, 7, dL, None)
    on = np.zeros(D.shape, bool)
    on[I, :] = True
    on[:, J] = True
    assert np.all(G[~on] == 0.0)
    assert np.abs(G[on]).max() > 0.0
    # the S output: outside rows I and columns J the gradient is exactly mask(S) * dS
    dS = rng.standard_normal(D.shape)
    G2 = adj.unrolled_vjp(D, I, J, 3, z0, 0.7, 7, None, dS)
    _, S = adj.unrolled_outputs(D, I, J, 3, z0, 0.7, 7)
    ms = adj.masks(D, I, J, 3, z0, 0.7, 7)[-1]
    assert np.array_equal(G2[~on], (ms * dS)[~on])
    assert np.count_nonzero(S[~on]) == np.count_nonzero(ms[~on])


def test_one_step_without_outliers_is_the_cur_formula():
    D, I, J = _case(seed=7)
    r = 3
    z0 = 1e6  # no residual exceeds zeta_0: T_zeta keeps nothing, S_1 = 0
    j = int(np.setdiff1d(np.arange(D.shape[1]), J)[0])
    dL = np.zeros(D.shape)
    rng = np.random.default_rng(2)
    dL[:, j] = rng.standard_normal(D.shape[0])
    G = adj.unrolled_vjp(D, I, J, r, z0, 0.7, 1, dL, None)
    # L(:, j) = C U^+ D(I, j) with C = D(:,J), U = H_r(D(I,J)): linear in D(I, j)
    W, s, Vt = np.linalg.svd(D[np.ix_(I, J)])
    Up = Vt[:r].T @ np.diag(1.0 / s[:r]) @ W[:, :r].T
    want = (D[:, J] @ Up).T @ dL[:, j]
    assert np.allclose(G[I, j], want, rtol=1e-10, atol=1e-12)
    rows_not_I = np.setdiff1d(np.arange(D.shape[0]), I)
    assert np.all(G[rows_not_I, j] == 0.0)


def test_final_keep_override():
    """final_keep replaces the last threshold's decisions only: with the FP64
    decisions themselves nothing changes; with one entry (i, j) outside rows I and
    columns J flipped, the gradient there becomes the flipped mask times dS_ij
    (D_ij enters the map nowhere else) and the L output is unchanged."""
    D, I, J = _case()
    r, T, g = 3, 5, 0.7
    z0 = float(np.abs(D).max())
    rng = np.random.default_rng(8)
    dL = rng.standard_normal(D.shape)
    dS = rng.standard_normal(D.shape)
    keep = adj.masks(D, I, J, r, z0, g, T)[-1]
    G = adj.unrolled_vjp(D, I, J, r, z0, g, T, dL, dS)
    assert np.allclose(adj.unrolled_vjp(D, I, J, r, z0, g, T, dL, dS, final_keep=keep), G, rtol=0, atol=1e-12)
    rows = np.setdiff1d(np.arange(D.shape[0]), I)
    cols = np.setdiff1d(np.arange(D.shape[1]), J)
    i, j = int(rows[1]), int(cols[2])
    flipped = keep.copy()
    flipped[i, j] = not keep[i, j]
    G2 = adj.unrolled_vjp(D, I, J, r, z0, g, T, dL, dS, final_keep=flipped)
    assert G[i, j] == (dS[i, j] if keep[i, j] else 0.0)
    assert G2[i, j] == (dS[i, j] if flipped[i, j] else 0.0)
    with torch.no_grad():
        L1, _ = adj.unrolled_forward(torch.tensor(D), I, J, r, z0, g, T)
        L2, S2 = adj.unrolled_forward(torch.tensor(D), I, J, r, z0, g, T, flipped)
    assert torch.equal(L1, L2)
    assert bool(S2[i, j] != 0) == bool(flipped[i, j])
