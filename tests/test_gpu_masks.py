"""Threshold-mask parity with the FP64 oracle, entry by entry (T_zeta, Sec. 3.2).

At iteration K the row panel keeps S_K(I,:) = T_zeta_K(D(I,:) - L_{K-1}(I,:))
and the column panel S_K(:,J) likewise.  The GPU's panels of iteration K come
through the C ABI (ircur_get_cur: C = [D - S_K]_{:,J}, R = [D - S_K]_{I,:}, so
an entry is thresholded exactly where it differs from D); the oracle's from its
history.  Both must take the same decision at every entry outside a tie band
around zeta_K.  The band at an entry is what the two iterates L_{K-1} may
differ by there (four times their measured difference) plus the FP32 rounding
of one evaluation of the rank-r product (64 u_fp32 (|D| + sum_t |A_it B_tj|)):
outside it, |D - L| - zeta has the same sign for both iterates.  Entries inside
the band are counted and reported, not failed (the tie reading of the threshold
operator).

Also checked: the index sets (IRCUR-R draws a new pair each iteration), the
(I,J) block read by both panels (bit-identical C(I,:) = R(:,J)), and that the
panel passes used the decisions get_cur reports (C U^+ R of those panels equals
the factors A_K B_K the passes wrote).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2010_07422_gb300 import ircur as ir  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402

U32 = 2.0 ** -24


def _gpu_run(D_t, n1, n2, r, K, resample, seed):
    s = ir.IRCUR(n1, n2, r, gamma=0.7, tol=1e-30, max_iter=K, resample=resample, seed=seed)
    res = s.solve(D_t)
    assert res.iters == K
    return s, res


def _factors64(s):
    A, B = s.factors()
    torch.cuda.synchronize()
    return A.double().cpu().numpy(), B.double().cpu().numpy()


def _band(D, L_g, L_o, A, B, rows, cols):
    """Per-entry tie band on the block D[rows][:, cols]."""
    absAB = np.abs(A[rows]) @ np.abs(B[:, cols])
    return 4.0 * np.abs(L_g - L_o) + 64.0 * U32 * (np.abs(D) + absAB) + 1e-30


def _check_iteration(p, D_t, r, K, resample, seed, hist, report):
    n1, n2 = p.D.shape
    D64 = p.D.astype(np.float64)
    h = hist[K - 1]
    I, J, zeta = h["I"], h["J"], h["zeta"]
    # the GPU at iteration K
    sK, resK = _gpu_run(D_t, n1, n2, r, K, resample, seed)
    Ig, Jg, _ = sK.indices()
    assert np.array_equal(Ig.cpu().numpy(), I) and np.array_equal(Jg.cpu().numpy(), J)
    Cg, Ug, Rg = sK.cur(D_t)
    torch.cuda.synchronize()
    Cg = Cg.double().cpu().numpy()
    Ug = Ug.double().cpu().numpy()
    Rg = Rg.double().cpu().numpy()
    AK, BK = _factors64(sK)
    sK.close()
    # the (I,J) block is the same FP32 value in both panels
    assert np.array_equal(Cg[I, :], Rg[:, J])
    mR_g = Rg != D64[I, :]
    mC_g = Cg != D64[:, J]
    mR_o = h["S_rows"] != 0
    mC_o = h["S_cols"] != 0
    # the iterate L_{K-1} on these panels: oracle (literal triple product) and GPU factors
    if K == 1:
        Lr_o = np.zeros((I.size, n2))
        Lc_o = np.zeros((n1, J.size))
        A1 = np.zeros((n1, r))
        B1 = np.zeros((r, n2))
    else:
        q = hist[K - 2]
        Lr_o = q["C"][I, :] @ q["U_pinv"] @ q["R"]
        Lc_o = q["C"] @ q["U_pinv"] @ q["R"][:, J]
        sP, _ = _gpu_run(D_t, n1, n2, r, K - 1, resample, seed)
        A1, B1 = _factors64(sP)
        sP.close()
    Lr_g = A1[I] @ B1
    Lc_g = A1 @ B1[:, J]
    allc = np.arange(n2)
    allr = np.arange(n1)
    bR = _band(D64[I, :], Lr_g, Lr_o, A1, B1, I, allc)
    bC = _band(D64[:, J], Lc_g, Lc_o, A1, B1, allr, J)
    gR = np.abs(np.abs(D64[I, :] - Lr_o) - zeta)
    gC = np.abs(np.abs(D64[:, J] - Lc_o) - zeta)
    outR, outC = gR > bR, gC > bC
    badR = int(np.sum((mR_g != mR_o) & outR))
    badC = int(np.sum((mC_g != mC_o) & outC))
    in_band = int(np.sum(~outR) + np.sum(~outC))
    total = mR_o.size + mC_o.size
    kept = int(mR_o.sum() + mC_o.sum())
    report.append((K, kept, in_band, badR + badC))
    assert badR == 0 and badC == 0, (K, badR, badC, in_band)
    assert in_band <= 1e-3 * total, (K, in_band, total)
    # the passes used these decisions: C U^+ R on the panels equals A_K B_K there
    Up = np.linalg.pinv(Ug, rcond=1e-6)
    L_cur_rows = Cg[I, :] @ Up @ Rg
    L_fac_rows = AK[I] @ BK
    assert np.linalg.norm(L_cur_rows - L_fac_rows) <= 1e-5 * np.linalg.norm(L_fac_rows)
    return kept


@pytest.mark.parametrize("n,Ks", [(1000, [1, 2, 3, 5, 8, 13, 20]), (10000, [2, 7, 14])])
@pytest.mark.parametrize("resample", [True, False])
def test_threshold_masks_match_the_oracle(n, Ks, resample):
    r, seed = 5, 9
    p = synth.planted(n, n, r, 0.1, seed=n + int(resample))
    ref = oracle.ircur(p.D, r, 0, 0.7, 1e-30, max(Ks), resample=resample, seed=seed, keep_history=True)
    D_t = torch.from_numpy(p.D).cuda()
    report = []
    for K in Ks:
        kept = _check_iteration(p, D_t, r, K, resample, seed, ref.history, report)
        if K == 1:
            assert kept == 0  # zeta_0 = max|D| thresholds nothing
        if K >= 3:
            assert kept > 0
    print("\n(K, thresholded entries, entries in the tie band, mismatches outside it):", report)


@pytest.mark.parametrize("resample", [True, False])
def test_final_sparse_support_matches_the_oracle(resample):
    """The dense outputs at tol = 1e-5: supp S = supp T_zeta(D - L) agrees with the
    oracle's outside the tie band of the two final L."""
    n, r, seed = 1000, 5, 4
    p = synth.planted(n, n, r, 0.1, seed=77)
    ref = oracle.ircur(p.D, r, 0, 0.7, 1e-5, 100, resample=resample, seed=seed)
    Lo, So = oracle.dense_outputs(p.D, ref)
    D_t = torch.from_numpy(p.D).cuda()
    s, res = _gpu_run(D_t, n, n, r, ref.iters, resample, seed)
    L, S = s.reconstruct(D_t)
    A, B = _factors64(s)
    s.close()
    Lg = L.double().cpu().numpy()
    Sg = S.double().cpu().numpy()
    D64 = p.D.astype(np.float64)
    band = _band(D64, Lg, Lo, A, B, np.arange(n), np.arange(n))
    out = np.abs(np.abs(D64 - Lo) - ref.zeta_next) > band
    mism = int(np.sum(((Sg != 0) != (So != 0)) & out))
    in_band = int(np.sum(~out))
    print(f"\nsupport of S: {int((So != 0).sum())} entries, {in_band} in the tie band, {mism} mismatches outside")
    assert mism == 0
    assert in_band <= 1e-4 * n * n
    # the planted support itself is found
    true_supp = np.zeros(n * n, bool)
    true_supp[p.s_pos] = True
    assert np.mean((Sg.reshape(-1) != 0) == true_supp) >= 0.999
