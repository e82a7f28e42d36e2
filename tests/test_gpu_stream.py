"""Streaming extension (ircur_stream_columns) against the FP64 oracle
(oracle.stream_columns, pinned in test_stream_oracle.py): new columns of the
same planted model, after a solve on the training columns.  The GPU and the
oracle each use their own model (the GPU's factors A, Y; the oracle's C, U^+)
from solves of the same D at the oracle's iteration count; bar 1e-5 relative
Frobenius on L and S, as for the solve itself.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2010_07422_gb300 import ircur as ir  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402

TOL = 1e-5


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def setup(n1, n2, c, r, alpha, resample, seed, **kw):
    p = synth.planted(n1, n2 + c, r, alpha, seed=seed)
    D = np.ascontiguousarray(p.D[:, :n2])
    Dn = np.ascontiguousarray(p.D[:, n2:])
    ref = oracle.ircur(D, r, 0.0, 0.7, 1e-5, 100, resample=resample, seed=seed, nI=kw.get("nI"), nJ=kw.get("nJ"))
    s = ir.IRCUR(n1, n2, r, tol=1e-12, max_iter=ref.iters, resample=resample, seed=seed, **kw)
    res = s.solve(torch.from_numpy(D).cuda())
    assert res.iters == ref.iters
    return p, D, Dn, ref, s


@pytest.mark.parametrize("n1,n2,c,r,alpha,resample,iters", [
    (1200, 1000, 64, 5, 0.1, False, 0),
    (1200, 1000, 64, 5, 0.1, True, 0),
    (900, 777, 33, 1, 0.05, True, 0),
    (1000, 1100, 100, 7, 0.15, False, 0),
    (800, 640, 40, 3, 0.1, False, 5),
    (700, 700, 1, 4, 0.1, True, 0),
])
def test_stream_matches_oracle(n1, n2, c, r, alpha, resample, iters):
    p, D, Dn, ref, s = setup(n1, n2, c, r, alpha, resample, seed=11 + r)
    K = iters or ref.iters
    Lo, So = oracle.stream_columns(Dn, ref, ref.zetas[0], 0.7, K)
    L, S = s.stream_columns(torch.from_numpy(Dn).cuda(), iters=iters)
    Lg, Sg = L.double().cpu().numpy(), S.double().cpu().numpy()
    assert rel(Lg, Lo) <= TOL, rel(Lg, Lo)
    assert rel(Sg, So) <= TOL, rel(Sg, So)
    if not iters:  # with the solve's iteration count the new columns' planted part is recovered
        Lt = (p.W @ p.V.T)[:, n2:]
        assert rel(Lg, Lt) <= 1e-3
    s.close()


def test_stream_rank_20():
    """r = 20 with |I| = |J| = 277: the streamed columns against the oracle."""
    n1, n2, c, r = 1000, 900, 50, 20
    p, D, Dn, ref, s = setup(n1, n2, c, r, 0.1, False, seed=31, nI=277, nJ=277)
    Lo, So = oracle.stream_columns(Dn, ref, ref.zetas[0], 0.7, ref.iters)
    L, S = s.stream_columns(torch.from_numpy(Dn).cuda())
    assert rel(L.double().cpu().numpy(), Lo) <= TOL
    assert rel(S.double().cpu().numpy(), So) <= TOL
    s.close()


def test_stream_padded_layout_and_no_sparse():
    n1, n2, c, r = 600, 500, 20, 3
    p, D, Dn, ref, s = setup(n1, n2, c, r, 0.1, False, seed=5)
    Lo, _ = oracle.stream_columns(Dn, ref, ref.zetas[0], 0.7, ref.iters)
    buf = torch.zeros(n1, c + 7, device="cuda")
    buf[:, :c] = torch.from_numpy(Dn).cuda()
    L, S = s.stream_columns(buf[:, :c], with_sparse=False)
    assert S is None
    assert rel(L.double().cpu().numpy(), Lo) <= TOL
    s.close()


def test_stream_errors():
    s = ir.IRCUR(300, 280, 2, resample=False)
    Dn = torch.zeros(300, 4, device="cuda")
    with pytest.raises(ir.IrcurError) as e:
        s.stream_columns(Dn)
    assert e.value.status == ir.IRCUR_ESTATE
    s.solve(torch.from_numpy(synth.planted(300, 280, 2, 0.1, seed=1).D).cuda())
    L = torch.zeros(300, 4, device="cuda")
    with pytest.raises(ir.IrcurError) as e:  # ldL < ncols
        ir.ircur_stream_columns(s._ctx, Dn, 4, 4, 0, L, 3)
    assert e.value.status == ir.IRCUR_EINVAL
    s.close()
