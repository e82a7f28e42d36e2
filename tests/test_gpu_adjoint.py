"""Adjoint of unrolled IRCUR-F (ircur_set_record / ircur_backward) against the
FP64 oracle gradient (oracle/ircur_adjoint.py, itself pinned by central finite
differences in test_adjoint_oracle.py).

Bar: relative Frobenius error of dD <= 1e-5.  The GPU path is FP32 with the
same index sets and the same threshold decisions as the oracle (the masks
themselves are compared with the oracle's entry by entry, outside a tie band, in
test_gpu_masks.py; an entry whose decision flipped would change the gradient far
beyond the bar); the error budget is FP32 rounding carried through K
iterations of rank-r products and the shifted conjugate-gradient solves
(stopped at 1e-6 relative residual), measured at 2e-7 .. 8e-7.

The last threshold, S = T_zeta_K(D - L_K) over all n1 n2 entries, can meet a
tie: an entry whose |D - L_K| is within FP32 rounding of zeta_K (at n = 4096 one
entry lies 1.5e-8 mean|D| from it), where the GPU and the FP64 oracle may take
different sides and one flip moves the gradient by about |dS_ij| / ||dD||.
There the oracle gradient is taken with the GPU's decisions (the tie reading of
T_zeta, Sec. 3.2), after checking that every decision that differs lies inside
the tie band of test_gpu_masks.py.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import ircur_adjoint as adj  # noqa: E402
from paper_2010_07422_gb300 import ircur as ir  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402

TOL_GRAD = 1e-5
U32 = 2.0 ** -24


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def setup(n1, n2, r, T, alpha, seed, **kw):
    p = synth.planted(n1, n2, r, alpha, seed=seed)
    D = torch.from_numpy(p.D).cuda()
    s = ir.IRCUR(n1, n2, r, tol=1e-12, max_iter=T, resample=False, seed=seed, **kw)
    s.record(True)
    res = s.solve(D)
    I = oracle.sample_indices(seed, 0, 0, n1, s.nI)
    J = oracle.sample_indices(seed, 0, 1, n2, s.nJ)
    return p, D, s, res, I, J


def gpu_final_keep(p, D, s, I, J, r, T, zeta0):
    """The GPU's decisions |D - A_K B_K| > zeta_K of the last threshold (the
    reconstruction kernel evaluates them with the backward's arithmetic) and the
    number that differ from the FP64 oracle's; each of those must lie in the tie
    band 4 |L_gpu - L_oracle| + 64 u (|D| + sum_t |A_it B_tj|)."""
    _, S = s.reconstruct(D)
    A, B = s.factors()
    torch.cuda.synchronize()
    keep = (S != 0).cpu().numpy()
    A = A.double().cpu().numpy()
    B = B.double().cpu().numpy()
    D64 = p.D.astype(np.float64)
    Lo, _ = adj.unrolled_outputs(D64, I, J, r, zeta0, 0.7, T)
    zT = zeta0 * 0.7 ** T
    ii, jj = np.nonzero(keep != (np.abs(D64 - Lo) > zT))
    if ii.size:
        lg = np.einsum("kt,tk->k", A[ii], B[:, jj])
        ab = np.einsum("kt,tk->k", np.abs(A[ii]), np.abs(B[:, jj]))
        d = D64[ii, jj]
        band = 4.0 * np.abs(lg - Lo[ii, jj]) + 64.0 * U32 * (np.abs(d) + ab)
        gap = np.abs(np.abs(d - Lo[ii, jj]) - zT)
        assert np.all(gap <= band), (ii, jj, gap, band)
    assert ii.size <= 1e-6 * keep.size, ii.size
    return keep, int(ii.size)


@pytest.mark.parametrize("n1,n2,r,T,alpha,seed,which", [
    (300, 260, 3, 6, 0.1, 1, "both"),
    (300, 260, 3, 6, 0.1, 1, "L"),
    (300, 260, 3, 6, 0.1, 1, "S"),
    (517, 333, 7, 10, 0.1, 2, "both"),
    (450, 470, 11, 8, 0.05, 3, "both"),   # padded rank 12
    (1024, 1024, 10, 15, 0.1, 4, "both"),  # the unrolled-training shape at n = 1024
    (200, 640, 1, 4, 0.2, 5, "both"),
])
def test_backward_matches_oracle_gradient(n1, n2, r, T, alpha, seed, which):
    p, D, s, res, I, J = setup(n1, n2, r, T, alpha, seed)
    assert res.iters == T and res.flags == 0
    rng = np.random.default_rng(seed)
    dL = rng.standard_normal((n1, n2)).astype(np.float32) if which in ("both", "L") else None
    dS = rng.standard_normal((n1, n2)).astype(np.float32) if which in ("both", "S") else None
    g = s.backward(D, None if dL is None else torch.from_numpy(dL).cuda(),
                   None if dS is None else torch.from_numpy(dS).cuda())
    keep, _ = gpu_final_keep(p, D, s, I, J, r, T, res.zeta0)
    G = adj.unrolled_vjp(p.D.astype(np.float64), I, J, r, res.zeta0, 0.7, T, dL, dS, final_keep=keep)
    gn = g.double().cpu().numpy()
    assert rel(gn, G) <= TOL_GRAD, rel(gn, G)
    on = np.zeros((n1, n2), bool)
    on[I, :] = True
    on[:, J] = True
    # outside rows I and columns J only the S output contributes, exactly mask(S) dS
    assert np.array_equal(gn[~on], G[~on])
    s.close()


def test_backward_rank_20():
    """r = 18 (padded rank 20) with |I| = |J| = 240: the same gradient parity."""
    n1, n2, r, T, seed = 600, 560, 18, 5, 6
    p, D, s, res, I, J = setup(n1, n2, r, T, 0.1, seed, nI=240, nJ=240)
    assert res.iters == T and res.flags & ~ir.IRCUR_FLAG_SVD_GAP == 0
    rng = np.random.default_rng(seed)
    dL = rng.standard_normal((n1, n2)).astype(np.float32)
    dS = rng.standard_normal((n1, n2)).astype(np.float32)
    g = s.backward(D, torch.from_numpy(dL).cuda(), torch.from_numpy(dS).cuda())
    keep, _ = gpu_final_keep(p, D, s, I, J, r, T, res.zeta0)
    G = adj.unrolled_vjp(p.D.astype(np.float64), I, J, r, res.zeta0, 0.7, T, dL, dS, final_keep=keep)
    assert rel(g.double().cpu().numpy(), G) <= TOL_GRAD, rel(g.double().cpu().numpy(), G)
    s.close()


def test_backward_at_training_size_properties():
    """n = 4096, r = 10, T = 15, |I| = |J| = ceil(40 ln 4096) = 333: the gradient of
    <dL, L> is supported on rows I and columns J, is finite, and is linear in dL."""
    n, r, T = 4096, 10, 15
    D = synth.planted_device(n, n, r, 0.1, seed=11)
    s = ir.IRCUR(n, n, r, tol=1e-12, max_iter=T, resample=False, seed=11)
    s.record(True)
    res = s.solve(D)
    assert res.iters == T and res.flags == 0
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    dL = torch.randn(n, n, device="cuda", generator=g)
    g1 = s.backward(D, dL, None)
    g2 = s.backward(D, 2.0 * dL, None)
    I, J, _ = s.indices()
    on = torch.zeros(n, n, dtype=torch.bool, device="cuda")
    on[I.long(), :] = True
    on[:, J.long()] = True
    assert torch.isfinite(g1).all()
    assert float(g1[~on].abs().max()) == 0.0
    assert float(g1[on].abs().max()) > 0.0
    assert float((g2 - 2.0 * g1).abs().max()) <= 1e-5 * float(g1.abs().max())
    s.close()


def test_backward_at_training_size_matches_oracle():
    """The unrolled-training shape itself: n = 4096, r = 10, T = 15 (|I| = |J| = 333),
    alpha = 0.1, cotangents for L and S: the GPU gradient against the FP64 oracle
    gradient, entry for entry, in relative Frobenius norm."""
    n, r, T, seed = 4096, 10, 15, 11
    p, D, s, res, I, J = setup(n, n, r, T, 0.1, seed)
    assert res.iters == T and res.flags == 0
    rng = np.random.default_rng(seed)
    dL = rng.standard_normal((n, n)).astype(np.float32)
    dS = rng.standard_normal((n, n)).astype(np.float32)
    g = s.backward(D, torch.from_numpy(dL).cuda(), torch.from_numpy(dS).cuda())
    torch.cuda.synchronize()
    gn = g.double().cpu().numpy()
    keep, ties = gpu_final_keep(p, D, s, I, J, r, T, res.zeta0)
    s.close()
    G = adj.unrolled_vjp(p.D.astype(np.float64), I, J, r, res.zeta0, 0.7, T, dL, dS, final_keep=keep)
    print(f"\nfinal-threshold ties taken on the GPU's side: {ties}")
    assert rel(gn, G) <= TOL_GRAD, rel(gn, G)


def test_backward_after_another_solve_is_refused():
    """The autograd Function holds the solver, whose recording belongs to its last
    solve: a solve between forward and backward makes backward raise ESTATE
    instead of differentiating the other solve."""
    n1, n2, r = 300, 280, 3
    p = synth.planted(n1, n2, r, 0.1, seed=41)
    D = torch.from_numpy(p.D).cuda().requires_grad_(True)
    s = ir.IRCUR(n1, n2, r, tol=1e-12, max_iter=5, resample=False, seed=41)
    L, S = ir.ircur_unrolled(D, s)
    s.solve(D.detach() * 2.0)
    with pytest.raises(ir.IrcurError) as e:
        (L.sum() + S.sum()).backward()
    assert e.value.status == ir.IRCUR_ESTATE
    L2, S2 = ir.ircur_unrolled(D, s)  # a fresh forward differentiates again
    (L2.sum() + S2.sum()).backward()
    assert torch.isfinite(D.grad).all()
    s.close()


def test_autograd_function_matches_direct_backward():
    n1, n2, r = 400, 380, 4
    p = synth.planted(n1, n2, r, 0.1, seed=21)
    Lt = torch.from_numpy(p.L_true()).float().cuda()
    D = torch.from_numpy(p.D).cuda().requires_grad_(True)
    s = ir.IRCUR(n1, n2, r, tol=1e-12, max_iter=8, resample=False, seed=21)
    L, S = ir.ircur_unrolled(D, s)
    lam = 0.1
    loss = ((L - Lt) ** 2).sum() + lam * S.abs().sum()
    loss.backward()
    dL = (2.0 * (L - Lt)).detach().contiguous()
    dS = (lam * torch.sign(S)).detach().contiguous()
    direct = s.backward(D.detach(), dL, dS)
    assert torch.allclose(D.grad, direct, rtol=1e-5, atol=1e-6 * float(direct.abs().max()))
    s.close()


def test_backward_errors():
    n1, n2, r = 200, 180, 2
    p = synth.planted(n1, n2, r, 0.1, seed=31)
    D = torch.from_numpy(p.D).cuda()
    s = ir.IRCUR(n1, n2, r, tol=1e-12, max_iter=3, resample=False, seed=31)
    s.solve(D)
    with pytest.raises(ir.IrcurError) as e:  # no recorded solve
        s.backward(D, torch.ones_like(D))
    assert e.value.status == ir.IRCUR_ESTATE
    s.record(True)
    with pytest.raises(ir.IrcurError) as e:  # recording on, no solve since
        s.backward(D, torch.ones_like(D))
    assert e.value.status == ir.IRCUR_ESTATE
    s.solve(D)
    s.backward(D, torch.ones_like(D))
    s.close()
    sr = ir.IRCUR(n1, n2, r, resample=True)
    with pytest.raises(ir.IrcurError) as e:  # IRCUR-R is not differentiated
        sr.record(True)
    assert e.value.status == ir.IRCUR_ENOTSUP
    sr.close()
