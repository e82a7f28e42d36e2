"""Algorithm 2 (CUR to SVD) on the GPU (ircur_get_svd) against the oracle's
Alg. 2 on the oracle's own C, U^+, R at the same iteration count.

Bars: singular values within 1e-5 relative; W, V orthonormal to 1e-5;
W diag(sigma) V^T equal to the GPU's own dense L to 1e-5 relative; each
singular vector equal to the oracle's up to sign (|<w, w_oracle>| >= 1 - 1e-4,
the singular values being distinct)."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2010_07422_gb300 import ircur as ir  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402


@pytest.mark.parametrize("n1,n2,r,alpha,resample", [
    (1000, 1000, 5, 0.1, True),
    (1000, 1000, 5, 0.1, False),
    (517, 333, 7, 0.1, False),
    (450, 470, 11, 0.05, True),   # padded rank 12
    (10000, 10000, 5, 0.1, True),  # the benchmark's size
])
def test_cur_to_svd_matches_oracle(n1, n2, r, alpha, resample, m=None):
    p = synth.planted(n1, n2, r, alpha, seed=n1 + r)
    ref = oracle.ircur(p.D, r, 0.0, 0.7, 1e-5, 100, resample=resample, seed=3, nI=m, nJ=m)
    Wo, so, Vo = oracle.cur_to_svd(ref.C, ref.U_pinv, ref.R)
    Wo, so, Vo = Wo[:, :r], so[:r], Vo[:, :r]
    D = torch.from_numpy(p.D).cuda()
    s = ir.IRCUR(n1, n2, r, nI=m or 0, nJ=m or 0, tol=1e-12, max_iter=ref.iters, resample=resample, seed=3)
    res = s.solve(D)
    assert res.iters == ref.iters
    W, sig, V = (t.double().cpu().numpy() for t in s.svd())
    assert np.all(np.diff(sig) <= 0)
    assert np.max(np.abs(sig - so) / so[0]) <= 1e-5, (sig, so)
    assert np.abs(W.T @ W - np.eye(r)).max() <= 1e-5
    assert np.abs(V.T @ V - np.eye(r)).max() <= 1e-5
    if n1 * n2 <= 1_000_000:
        L, _ = s.reconstruct(D, with_sparse=False)
        L = L.double().cpu().numpy()
        assert np.linalg.norm((W * sig) @ V.T - L) <= 1e-5 * np.linalg.norm(L)
    assert np.all(np.abs(np.sum(W * Wo, axis=0)) >= 1 - 1e-4)
    assert np.all(np.abs(np.sum(V * Vo, axis=0)) >= 1 - 1e-4)
    s.close()


def test_cur_to_svd_rank_20():
    """r = 20 (Fig. 1's third rank) with |I| = |J| = 277 at n = 1000."""
    test_cur_to_svd_matches_oracle(1000, 1000, 20, 0.1, True, m=277)


def test_cur_to_svd_needs_a_solve():
    s = ir.IRCUR(200, 180, 2)
    with pytest.raises(ir.IrcurError) as e:
        s.svd()
    assert e.value.status == ir.IRCUR_ESTATE
    s.close()
