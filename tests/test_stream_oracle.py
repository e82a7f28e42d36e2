"""Pins of the streaming oracle (oracle.stream_columns): new columns against a
fixed CUR model.  Closed forms only:
* a pure low-rank D gives an exact model (Thm 1: C U^+ R = D), and then every
  new column in the column space is reproduced exactly with S = 0;
* the same column with outliers larger than zeta_0 on a few rows (inside and
  outside I) comes back as L = the low-rank column and S = the outliers;
* scaling the columns and zeta_0 by a power of two scales L and S exactly.
"""

import numpy as np

import oracle


def exact_model(n1=300, n2=280, r=3, seed=0):
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((n1, r))
    V = rng.standard_normal((n2, r))
    D = W @ V.T
    res = oracle.ircur(D, r, 0.0, 0.7, 1e-12, 5, seed=seed)
    return W, D, res


def test_columns_in_the_span_are_reproduced():
    W, D, res = exact_model()
    assert res.iters == 1 and res.errs[-1] < 1e-12
    v = np.random.default_rng(1).standard_normal((W.shape[1], 40))
    d = W @ v
    zeta0 = res.zetas[0]
    L, S = oracle.stream_columns(d, res, zeta0, 0.7, 10)
    assert np.max(np.abs(L - d)) <= 1e-9 * np.max(np.abs(d))
    assert not np.any(S)


def test_outliers_are_separated():
    W, D, res = exact_model(seed=2)
    rng = np.random.default_rng(3)
    c = 12
    low = W @ rng.standard_normal((W.shape[1], c))
    spikes = np.zeros_like(low)
    big = 3.0 * float(np.max(np.abs(D)))  # above zeta_0 = max|D|: thresholded from the first step
    for q in range(c):
        rows = rng.choice(W.shape[0], 4, replace=False)
        rows[0] = res.I[q % len(res.I)]  # at least one outlier on a sampled row
        spikes[rows, q] = big * np.where(rng.random(4) < 0.5, -1.0, 1.0)
    L, S = oracle.stream_columns(low + spikes, res, res.zetas[0], 0.7, 30)
    scale = float(np.max(np.abs(low)))
    assert np.max(np.abs(L - low)) <= 1e-9 * scale
    assert np.max(np.abs(S - spikes)) <= 1e-9 * scale
    assert np.array_equal(S != 0, spikes != 0)


def test_power_of_two_scaling_is_exact():
    W, D, res = exact_model(seed=4)
    rng = np.random.default_rng(5)
    d = W @ rng.standard_normal((W.shape[1], 6)) + (rng.random((W.shape[0], 6)) < 0.05) * 20.0
    L1, S1 = oracle.stream_columns(d, res, res.zetas[0], 0.7, 12)
    res2 = oracle.ircur(8.0 * D, W.shape[1], 0.0, 0.7, 1e-12, 5, seed=4)
    L2, S2 = oracle.stream_columns(8.0 * d, res2, res2.zetas[0], 0.7, 12)
    assert np.array_equal(L2, 8.0 * L1) and np.array_equal(S2, 8.0 * S1)


def test_single_column_and_iteration_count():
    W, D, res = exact_model(seed=6)
    d = W[:, 0] * 2.0
    L, S = oracle.stream_columns(d, res, res.zetas[0], 0.7, 1)
    assert L.shape == (W.shape[0], 1)
    # one step with zeta_0 = max|D| >= max|d_I| keeps every entry: L = C U^+ d_I
    want = oracle.cur_product(res.C, res.U_pinv, d[res.I][:, None])
    assert np.allclose(L, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_outliers_below_zeta0_need_the_iteration():
    """Outliers of 0.4 max|D| are kept by the first threshold and smeared into
    L_1; only the iteration (L_I updated, zeta decaying) separates them.  With
    L_I held at 0 the decaying threshold would cut the low-rank entries too."""
    W, D, res = exact_model(seed=8)
    rng = np.random.default_rng(9)
    c = 10
    low = W @ rng.standard_normal((W.shape[1], c))
    spikes = np.zeros_like(low)
    mag = 0.4 * float(np.max(np.abs(D)))
    for q in range(c):
        rows = rng.choice(W.shape[0], 3, replace=False)
        rows[0] = res.I[(3 * q) % len(res.I)]
        spikes[rows, q] = mag * np.where(rng.random(3) < 0.5, -1.0, 1.0)
    L, S = oracle.stream_columns(low + spikes, res, res.zetas[0], 0.7, 40)
    scale = float(np.max(np.abs(low)))
    assert np.max(np.abs(L - low)) <= 1e-8 * scale
    assert np.array_equal(S != 0, spikes != 0)
    # one step only: the outliers on I are still inside L
    L1, _ = oracle.stream_columns(low + spikes, res, res.zetas[0], 0.7, 1)
    assert np.max(np.abs(L1 - low)) > 1e-3 * scale
