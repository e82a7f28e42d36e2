"""Batched solves of independent problems (ircur_batch_*), through the C ABI.

Each instance of a batch must compute what a lone solve of the same problem
computes, bit for bit (instances keep their own padded rank; the batch groups
them by it), and so stay within the parity bar against the FP64 oracle.
"""

import ctypes

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


def to_dev(D_np):
    return torch.from_numpy(np.ascontiguousarray(D_np, dtype=np.float32)).cuda()


def lone(D, q):
    s = ir.IRCUR(q["n1"], q["n2"], q["r"], nI=q.get("nI", 0), nJ=q.get("nJ", 0), zeta0=q.get("zeta0", 0.0),
                 gamma=q.get("gamma", 0.7), tol=q.get("tol", 1e-5), max_iter=q.get("max_iter", 100),
                 resample=q.get("resample", True), seed=q.get("seed", 0))
    res = s.solve(D)
    A, B = s.factors()
    L, S = s.reconstruct(D)
    torch.cuda.synchronize()
    out = (res, A.cpu().numpy(), B.cpu().numpy(), L.cpu().numpy(), S.cpu().numpy())
    s.close()
    return out


SAME_RANK = [
    dict(n1=300, n2=410, r=5, resample=True, seed=1, gamma=0.7, alpha=0.1),
    dict(n1=777, n2=512, r=5, resample=False, seed=2, gamma=0.65, alpha=0.2),
    dict(n1=1000, n2=1000, r=5, resample=True, seed=3, gamma=0.7, alpha=0.1),
    dict(n1=256, n2=900, r=5, resample=True, seed=4, gamma=0.8, alpha=0.05, max_iter=3),
    dict(n1=640, n2=333, r=5, resample=False, seed=5, gamma=0.7, alpha=0.15, nI=60, nJ=90),
    dict(n1=501, n2=499, r=5, resample=True, seed=6, gamma=0.6, alpha=0.1, tol=1e-3),
]


def test_batch_equals_lone_solves_bitwise():
    """Same padded rank everywhere: every instance matches its lone solve bit for bit
    (iterations, stopping value, factors, dense outputs), including an instance
    that hits its own iteration cap and one that stops at a looser tolerance
    while the others go on."""
    Ds = [to_dev(synth.planted(q["n1"], q["n2"], q["r"], q["alpha"], seed=10 + i).D)
          for i, q in enumerate(SAME_RANK)]
    probs = [{k: v for k, v in q.items() if k != "alpha"} for q in SAME_RANK]
    batch = ir.IRCURBatch(probs)
    got = batch.solve(Ds)
    iters = set()
    for i, (q, D) in enumerate(zip(probs, Ds)):
        res, A, B, L, S = lone(D, q)
        g = got[i]
        assert (g.iters, g.converged, g.flags, g.svd_steps) == (res.iters, res.converged, res.flags, res.svd_steps)
        assert g.final_err == res.final_err and g.zeta_next == res.zeta_next
        Ab, Bb = batch[i].factors()
        Lb, Sb = batch[i].reconstruct(D)
        assert np.array_equal(Ab.cpu().numpy(), A) and np.array_equal(Bb.cpu().numpy(), B)
        assert np.array_equal(Lb.cpu().numpy(), L) and np.array_equal(Sb.cpu().numpy(), S)
        iters.add(g.iters)
    assert got[3].iters == 3 and not got[3].converged
    assert len(iters) > 1  # the instances really stopped at different iterations
    batch.close()


MIXED = [
    dict(n1=333, n2=517, r=1, resample=True, seed=1, alpha=0.05),
    dict(n1=517, n2=333, r=7, resample=False, seed=2, alpha=0.1),
    dict(n1=450, n2=470, r=11, resample=True, seed=3, alpha=0.05),
    dict(n1=260, n2=830, r=2, resample=True, seed=4, alpha=0.1),
    dict(n1=600, n2=600, r=3, resample=False, seed=5, alpha=0.2),
]


def test_batch_mixed_ranks_match_oracle():
    """Ranks 1..11 in one batch (five rank groups): each instance against the
    FP64 oracle at the oracle's own iteration count, and bit for bit against
    its lone solve."""
    probs, Ds, refs, Dn = [], [], [], []
    for i, q in enumerate(MIXED):
        p = synth.planted(q["n1"], q["n2"], q["r"], q["alpha"], seed=100 + i)
        ref = oracle.ircur(p.D, q["r"], 0.0, 0.7, 1e-5, 100, resample=q["resample"], seed=q["seed"])
        refs.append(ref)
        Dn.append(p.D)
        Ds.append(to_dev(p.D))
        probs.append(dict(n1=q["n1"], n2=q["n2"], r=q["r"], resample=q["resample"], seed=q["seed"],
                          tol=1e-12, max_iter=ref.iters))
    batch = ir.IRCURBatch(probs)
    got = batch.solve(Ds)
    for i, ref in enumerate(refs):
        assert got[i].iters == ref.iters
        L, S = batch[i].reconstruct(Ds[i])
        Lo, So = oracle.dense_outputs(Dn[i], ref)
        assert rel(L.double().cpu().numpy(), Lo) <= TOL_LS, (i, rel(L.double().cpu().numpy(), Lo))
        assert rel(S.double().cpu().numpy(), So) <= TOL_LS, (i, rel(S.double().cpu().numpy(), So))
        q = probs[i]
        res_l, A_l, B_l, L_l, S_l = lone(Ds[i], q)
        assert got[i].iters == res_l.iters and got[i].final_err == res_l.final_err
        assert np.array_equal(L.cpu().numpy(), L_l) and np.array_equal(S.cpu().numpy(), S_l)
        I, J, _ = batch[i].indices()
        draw = ref.iters - 1 if MIXED[i]["resample"] else 0
        Iw = oracle.sample_indices(MIXED[i]["seed"], draw, 0, MIXED[i]["n1"], batch[i].nI)
        Jw = oracle.sample_indices(MIXED[i]["seed"], draw, 1, MIXED[i]["n2"], batch[i].nJ)
        assert np.array_equal(I.cpu().numpy(), Iw) and np.array_equal(J.cpu().numpy(), Jw)
    batch.close()


def test_batch_with_rank_20_group():
    """Ranks 3 and 20 (two rank groups: the two-phase iteration with the
    separate look-ahead draws), IRCUR-R and -F: each instance equals its lone
    solve bit for bit."""
    probs = [dict(n1=900, n2=800, r=20, nI=250, nJ=260, resample=True, seed=1),
             dict(n1=500, n2=700, r=3, resample=True, seed=2),
             dict(n1=820, n2=760, r=17, nI=230, nJ=230, resample=False, seed=3)]
    Ds = [to_dev(synth.planted(q["n1"], q["n2"], q["r"], 0.1, seed=40 + i).D) for i, q in enumerate(probs)]
    batch = ir.IRCURBatch([dict(q, tol=1e-5, max_iter=100) for q in probs])
    got = batch.solve(Ds)
    for i, (q, D) in enumerate(zip(probs, Ds)):
        res, A, B, L, S = lone(D, dict(q, tol=1e-5, max_iter=100))
        assert (got[i].iters, got[i].final_err) == (res.iters, res.final_err)
        Lb, Sb = batch[i].reconstruct(D)
        assert np.array_equal(Lb.cpu().numpy(), L) and np.array_equal(Sb.cpu().numpy(), S)
    batch.close()


def test_batch_replay_rebuild_and_host_loop(monkeypatch):
    """Replaying the recorded graph, recording a new one for new D pointers, and
    the host-driven loop all give the same results."""
    probs = [dict(n1=400, n2=300, r=3, seed=1), dict(n1=350, n2=380, r=4, resample=False, seed=2),
             dict(n1=200, n2=210, r=2, seed=3)]
    Ds = [to_dev(synth.planted(q["n1"], q["n2"], q["r"], 0.1, seed=20 + i).D) for i, q in enumerate(probs)]
    batch = ir.IRCURBatch(probs)

    def run(Dl):
        res = batch.solve(Dl)
        return [(r.iters, r.final_err) for r in res], [batch[i].factors()[1].cpu().numpy() for i in range(3)]

    first = run(Ds)
    again = run(Ds)
    moved = run([D.clone() for D in Ds])
    monkeypatch.setenv("IRCUR_NO_GRAPH", "1")
    host = run(Ds)
    for other in (again, moved, host):
        assert other[0] == first[0]
        for a, b in zip(other[1], first[1]):
            assert np.array_equal(a, b)
    batch.close()


def test_batch_errors():
    lib = ir._lib()
    P = ir.ircur_params
    good = P(n1=100, n2=100, r=2, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=10, resample=1, seed=0,
             precision=0, svd_form=0)
    bad = P(n1=100, n2=100, r=0, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=10, resample=1, seed=0,
            precision=0, svd_form=0)
    h = ctypes.c_void_p()
    assert lib.ircur_batch_create((P * 1)(good), 0, None, ctypes.byref(h)) == ir.IRCUR_EINVAL
    assert lib.ircur_batch_create((P * 2)(good, bad), 2, None, ctypes.byref(h)) == ir.IRCUR_EINVAL
    assert not h.value
    b = ir.ircur_batch_create([good, good])
    assert ir.ircur_batch_instance(b, 2).value is None
    assert ir.ircur_batch_instance(b, -1).value is None
    D = torch.zeros(100, 100, device="cuda")
    status, _ = ir.ircur_batch_solve(b, [D, D], [100, 99])
    assert status == ir.IRCUR_EINVAL
    # getters before a solve
    assert lib.ircur_get_factors(ir.ircur_batch_instance(b, 0), None, None) == ir.IRCUR_ESTATE
    status, res = ir.ircur_batch_solve(b, [D, D], [100, 100])
    assert status == ir.IRCUR_OK
    ir.ircur_batch_destroy(b)
