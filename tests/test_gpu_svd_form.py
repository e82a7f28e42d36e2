"""The one-CTA form of the core SVD (svd_form = IRCUR_SVD_ONE_CTA) through the
C ABI: parity with the FP64 oracle at the oracle's iteration count (the same
1e-5 bar as the cluster form), agreement of the two forms, the fallback to
the cluster form where the core does not fit one SM, and batches of one-CTA
instances equal to lone one-CTA solves bit for bit.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2010_07422_gb300 import ircur as ir  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402

TOL_LS = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def solve(D_np, r, form, **kw):
    n1, n2 = D_np.shape
    D = torch.from_numpy(np.ascontiguousarray(D_np, np.float32)).cuda()
    s = ir.IRCUR(n1, n2, r, svd_form=form, **kw)
    res = s.solve(D)
    L, S = s.reconstruct(D)
    A, B = s.factors()
    torch.cuda.synchronize()
    out = (res, L.double().cpu().numpy(), S.double().cpu().numpy(), A.cpu().numpy(), B.cpu().numpy())
    s.close()
    return out


CASES = [
    # n1, n2, r, alpha, resample, nI, nJ   (the last two: core 230 x 230 does not fit: cluster fallback)
    (1000, 1000, 5, 0.1, True, 0, 0),
    (1000, 1000, 5, 0.2, False, 0, 0),
    (777, 512, 1, 0.1, True, 0, 0),
    (640, 901, 3, 0.1, False, 90, 150),
    (900, 700, 7, 0.05, True, 0, 0),
    (800, 820, 8, 0.1, True, 150, 160),
    (1200, 1100, 6, 0.1, True, 230, 230),
]


@pytest.mark.parametrize("n1,n2,r,alpha,resample,nI,nJ", CASES)
def test_one_cta_matches_oracle(n1, n2, r, alpha, resample, nI, nJ):
    p = synth.planted(n1, n2, r, alpha, seed=7)
    ref = oracle.ircur(p.D, r, 0.0, 0.7, 1e-5, 100, nI=nI or None, nJ=nJ or None, resample=resample, seed=3)
    K = ref.iters
    got = solve(p.D, r, ir.IRCUR_SVD_ONE_CTA, nI=nI, nJ=nJ, tol=1e-12, max_iter=K, resample=resample, seed=3)
    Lo, So = oracle.dense_outputs(p.D, ref)
    assert got[0].iters == K and got[0].flags == 0
    assert rel(got[1], Lo) <= TOL_LS, rel(got[1], Lo)
    assert rel(got[2], So) <= TOL_LS, rel(got[2], So)
    cl = solve(p.D, r, ir.IRCUR_SVD_CLUSTER, nI=nI, nJ=nJ, tol=1e-12, max_iter=K, resample=resample, seed=3)
    assert rel(got[1], cl[1]) <= TOL_LS
    if nI > 200:  # no one-CTA core of this size: the cluster form ran, bit for bit
        assert all(np.array_equal(a, b) for a, b in zip(got[1:], cl[1:]))


def test_one_cta_deterministic():
    p = synth.planted(1000, 1000, 5, 0.1, seed=9)
    a = solve(p.D, 5, ir.IRCUR_SVD_ONE_CTA, tol=1e-12, max_iter=15, seed=1)
    b = solve(p.D, 5, ir.IRCUR_SVD_ONE_CTA, tol=1e-12, max_iter=15, seed=1)
    assert a[0].svd_steps == b[0].svd_steps
    assert all(np.array_equal(x, y) for x, y in zip(a[1:], b[1:]))


def test_batch_of_one_cta_instances_equals_lone_solves():
    qs = [dict(n1=500, n2=610, r=5, resample=True, seed=1, svd_form=1),
          dict(n1=700, n2=450, r=2, resample=False, seed=2, svd_form=1),
          dict(n1=620, n2=600, r=8, resample=True, seed=3, svd_form=1),
          dict(n1=640, n2=530, r=5, resample=True, seed=4, svd_form=0),   # cluster form in the same group
          dict(n1=660, n2=540, r=5, resample=True, seed=6, svd_form=2),   # cluster of 8 in the same group
          dict(n1=1200, n2=1100, r=6, nI=230, nJ=230, resample=True, seed=5, svd_form=1)]  # falls back
    Ds = [torch.from_numpy(synth.planted(q["n1"], q["n2"], q["r"], 0.1, seed=30 + i).D).cuda()
          for i, q in enumerate(qs)]
    batch = ir.IRCURBatch(qs)
    got = batch.solve(Ds)
    for i, (q, D) in enumerate(zip(qs, Ds)):
        s = ir.IRCUR(q["n1"], q["n2"], q["r"], nI=q.get("nI", 0), nJ=q.get("nJ", 0), resample=q["resample"],
                     seed=q["seed"], svd_form=q["svd_form"])
        res = s.solve(D)
        A, B = s.factors()
        Ab, Bb = batch[i].factors()
        assert (got[i].iters, got[i].final_err, got[i].svd_steps) == (res.iters, res.final_err, res.svd_steps)
        assert torch.equal(A, Ab) and torch.equal(B, Bb)
        s.close()
    batch.close()


@pytest.mark.parametrize("resample", [True, False])
def test_cluster_of_8_matches_oracle(resample):
    """svd_form = IRCUR_SVD_CLUSTER8 (8 CTAs where the slabs of 8 fit): parity with
    the oracle at 1e-5 and agreement with the default cluster form."""
    p = synth.planted(1000, 1000, 5, 0.1, seed=7)
    ref = oracle.ircur(p.D, 5, 0.0, 0.7, 1e-5, 100, resample=resample, seed=3)
    K = ref.iters
    got = solve(p.D, 5, ir.IRCUR_SVD_CLUSTER8, tol=1e-12, max_iter=K, resample=resample, seed=3)
    Lo, So = oracle.dense_outputs(p.D, ref)
    assert got[0].iters == K and got[0].flags == 0
    assert rel(got[1], Lo) <= TOL_LS, rel(got[1], Lo)
    assert rel(got[2], So) <= TOL_LS, rel(got[2], So)
    cl = solve(p.D, 5, ir.IRCUR_SVD_CLUSTER, tol=1e-12, max_iter=K, resample=resample, seed=3)
    assert rel(got[1], cl[1]) <= TOL_LS
