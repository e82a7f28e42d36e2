"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars (stated by the method's accuracy target): relative Frobenius error of the
dense L and S <= 1e-5 for the FP32 path at equal iteration counts; index sets
bit-exact; stopping values e_k within 1e-3 relative of the oracle's (the FP32
residual floor is ~1e-7 of ||D||, far below the 1e-5 tolerance).
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


def gpu_solve(D_np, r, *, max_iter, tol=1e-12, resample=True, seed=0, nI=0, nJ=0, zeta0=0.0,
              gamma=0.7, idx=None, ld=None, offset=0):
    n1, n2 = D_np.shape
    ld = ld or n2
    buf = torch.zeros(n1 * ld + offset + 4, dtype=torch.float32, device="cuda")
    Dv = buf[offset:offset + n1 * ld].view(n1, ld)
    Dv[:, :n2] = torch.from_numpy(np.ascontiguousarray(D_np, dtype=np.float32)).cuda()
    D = Dv[:, :n2]
    s = ir.IRCUR(n1, n2, r, nI=nI, nJ=nJ, zeta0=zeta0, gamma=gamma, tol=tol, max_iter=max_iter,
                 resample=resample, seed=seed)
    if idx is not None:
        I_all, J_all = idx
        res = s.solve(D, torch.from_numpy(I_all.astype(np.int32)).cuda(),
                      torch.from_numpy(J_all.astype(np.int32)).cuda())
    else:
        res = s.solve(D)
    L, S = s.reconstruct(D)
    torch.cuda.synchronize()
    return s, res, L.double().cpu().numpy(), S.double().cpu().numpy()


def oracle_run(D_np, r, *, max_iter, tol=1e-12, resample=True, seed=0, nI=None, nJ=None, zeta0=0.0,
               gamma=0.7, draws=None):
    return oracle.ircur(D_np, r, zeta0, gamma, tol, max_iter, nI=nI, nJ=nJ, resample=resample, seed=seed,
                        index_draws=draws)


# ---------------------------------------------------------------- a1: sampler
@pytest.mark.parametrize("seed,draw,axis,n,m", [
    (0, 0, 0, 1000, 139), (1, 5, 1, 1000, 139), (123456789, 99, 0, 10000, 185),
    (7, 3, 1, 81920, 91), (2, 0, 0, 17, 17), (3, 1, 1, 5, 1), (2 ** 63 + 5, 7, 0, 3055, 65),
    (11, 2, 0, 333, 37),
])
def test_device_sampler_bit_exact(seed, draw, axis, n, m):
    got = ir.sample_indices(seed, draw, axis, n, m).cpu().numpy()
    want = oracle.sample_indices(seed, draw, axis, n, m)
    assert np.array_equal(got, want)


# ---------------------------------------------------------------- first iteration
def test_first_iteration_is_the_cur_of_D():
    """zeta_0 = max|D| keeps S_1 = 0, so L_1 = CUR(D) on the sampled sets."""
    p = synth.planted(500, 420, 4, 0.1, seed=1)
    ref = oracle_run(p.D, 4, max_iter=1, seed=3)
    s, res, L, S = gpu_solve(p.D, 4, max_iter=1, seed=3)
    assert res.iters == 1
    Lo, So = oracle.dense_outputs(p.D, ref)
    assert rel(L, Lo) <= TOL_LS and rel(S, So) <= TOL_LS
    assert abs(res.final_err - ref.errs[0]) <= 1e-4 * ref.errs[0]
    assert res.zeta0 == float(np.abs(p.D).max())


# ---------------------------------------------------------------- full loop, config-0 shape
@pytest.mark.parametrize("resample", [True, False])
def test_config0_parity(resample):
    """n = 1000, r = 5, alpha = 0.1, |I| = |J| = 139, zeta_0 = max|D|, gamma = 0.7, tol = 1e-5."""
    p = synth.planted(1000, 1000, 5, 0.1, seed=0)
    ref = oracle_run(p.D, 5, max_iter=100, tol=1e-5, resample=resample, seed=1)
    K = ref.iters
    # same iteration count as the oracle
    s, res, L, S = gpu_solve(p.D, 5, max_iter=K, resample=resample, seed=1)
    Lo, So = oracle.dense_outputs(p.D, ref)
    assert res.iters == K
    assert rel(L, Lo) <= TOL_LS, rel(L, Lo)
    assert rel(S, So) <= TOL_LS, rel(S, So)
    errs = np.array(s.errors())
    assert np.all(np.abs(errs[:5] - np.array(ref.errs[:5])) <= 1e-3 * np.array(ref.errs[:5]))
    # the stopping test itself: GPU at tol = 1e-5 stops within one iteration of the oracle
    s2, res2, L2, _ = gpu_solve(p.D, 5, max_iter=100, tol=1e-5, resample=resample, seed=1)
    assert res2.converged and abs(res2.iters - K) <= 1
    Lt = p.L_true()
    assert rel(L2, Lt) <= 1e-3  # the paper's success criterion (Sec. 4.1.1)
    assert res2.flags == 0


# ---------------------------------------------------------------- ragged shapes and ranks
@pytest.mark.parametrize("n1,n2,r,alpha,resample", [
    (333, 517, 1, 0.05, True),
    (517, 333, 7, 0.1, False),
    (450, 470, 11, 0.05, True),   # padded rank 12
    (390, 401, 16, 0.02, False),  # largest rank
    (260, 1030, 2, 0.1, True),
])
def test_ragged_shapes_parity(n1, n2, r, alpha, resample):
    p = synth.planted(n1, n2, r, alpha, seed=n1 + r)
    ref = oracle_run(p.D, r, max_iter=100, tol=1e-5, resample=resample, seed=2)
    K = ref.iters
    s, res, L, S = gpu_solve(p.D, r, max_iter=K, resample=resample, seed=2)
    Lo, So = oracle.dense_outputs(p.D, ref)
    assert res.iters == K
    assert rel(L, Lo) <= TOL_LS, rel(L, Lo)
    assert rel(S, So) <= TOL_LS, rel(S, So)


@pytest.mark.parametrize("n1,n2,r,m,resample", [
    (1000, 1000, 20, 277, True),   # r = 20 of Fig. 1: |I| = |J| = ceil(2 r ln n)
    (1000, 1000, 20, 415, False),  # c_I = 3: the largest rank-20 core that fits
    (700, 900, 17, 300, True),     # padded rank 20, ragged
])
def test_rank_20_parity(n1, n2, r, m, resample):
    p = synth.planted(n1, n2, r, 0.1, seed=n1 + r + m)
    ref = oracle_run(p.D, r, max_iter=100, tol=1e-5, resample=resample, seed=3, nI=m, nJ=m)
    K = ref.iters
    s, res, L, S = gpu_solve(p.D, r, max_iter=K, resample=resample, seed=3, nI=m, nJ=m)
    Lo, So = oracle.dense_outputs(p.D, ref)
    assert res.iters == K
    assert rel(L, Lo) <= TOL_LS, (rel(L, Lo), res.flags)
    assert rel(S, So) <= TOL_LS, (rel(S, So), res.flags)
    # no rank lost and no step cap; IRCUR_FLAG_SVD_GAP may report an early
    # core whose sigma_20 / sigma_21 was narrow (outliers not yet removed)
    assert res.flags & ~ir.IRCUR_FLAG_SVD_GAP == 0, res.flags


def test_rank_20_limits():
    """r = 21 is beyond the built ranks.  At r = 20 the core SVD's cluster of 16
    CTAs holds a 415 x 415 core (c_I = 3 at n = 1000) in shared memory, not a
    484 x 484 one (c_I = 3.5): ENOTSUP."""
    with pytest.raises(RuntimeError, match="ENOTSUP"):
        ir.IRCUR(1000, 1000, 21, nI=200, nJ=200)
    with pytest.raises(RuntimeError, match="ENOTSUP"):
        ir.IRCUR(1000, 1000, 20, nI=484, nJ=484)
    ir.IRCUR(1000, 1000, 20, nI=415, nJ=415).close()


def test_explicit_indices_padded_ld_and_unaligned_pointer():
    """Caller-supplied index sets (drawn by numpy), ldD > n2 and a D pointer
    that is 4- but not 16-byte aligned (the non-bulk row path)."""
    n1, n2, r, K = 300, 257, 3, 12
    p = synth.planted(n1, n2, r, 0.1, seed=4)
    nI, nJ = 60, 55
    I_all = np.stack([synth.random_subset(n1, nI, 100 + k) for k in range(K)])
    J_all = np.stack([synth.random_subset(n2, nJ, 200 + k) for k in range(K)])
    ref = oracle_run(p.D, r, max_iter=K, nI=nI, nJ=nJ, draws=lambda k: (I_all[k], J_all[k]))
    s, res, L, S = gpu_solve(p.D, r, max_iter=K, nI=nI, nJ=nJ, idx=(I_all, J_all), ld=263, offset=1)
    Lo, So = oracle.dense_outputs(p.D, ref)
    assert rel(L, Lo) <= TOL_LS and rel(S, So) <= TOL_LS


def test_fixed_zeta0_and_pure_low_rank():
    rng = np.random.default_rng(5)
    n1, n2, r = 400, 350, 4
    Dlr = (rng.standard_normal((n1, r)) @ rng.standard_normal((r, n2))).astype(np.float32)
    s, res, L, S = gpu_solve(Dlr, r, max_iter=20, tol=1e-5, zeta0=50.0)
    assert res.iters == 1 and res.converged and res.final_err < 1e-5
    assert rel(L, Dlr.astype(np.float64)) <= 1e-5
    assert res.zeta0 == 50.0


# ---------------------------------------------------------------- invariants
def test_deterministic_and_graph_equals_host_loop(monkeypatch):
    p = synth.planted(600, 600, 5, 0.1, seed=6)
    D = torch.from_numpy(p.D).cuda()
    outs = []
    for no_graph in ("0", "0", "1"):
        monkeypatch.setenv("IRCUR_NO_GRAPH", no_graph)
        s = ir.IRCUR(600, 600, 5, tol=1e-5, resample=True, seed=9)
        res = s.solve(D)
        A, B = s.factors()
        outs.append((res.iters, A.cpu().numpy(), B.cpu().numpy()))
        s.close()
    for o in outs[1:]:
        assert o[0] == outs[0][0]
        assert np.array_equal(o[1], outs[0][1]) and np.array_equal(o[2], outs[0][2])


def test_rank_and_scaling():
    p = synth.planted(500, 500, 3, 0.1, seed=8)
    _, res, L, _ = gpu_solve(p.D, 3, max_iter=60, tol=1e-5, seed=4)
    sv = np.linalg.svd(L, compute_uv=False)
    assert sv[3] <= 1e-5 * sv[0]
    # scaling D and zeta_0 by 4 scales L by 4 (the same masks)
    _, res4, L4, _ = gpu_solve(p.D * 4, 3, max_iter=res.iters, seed=4)
    assert rel(L4, 4 * L) <= 1e-6


def test_host_memory_entry_point_matches_device_path():
    p = synth.planted(700, 640, 4, 0.1, seed=9)
    s, res, L, S = gpu_solve(p.D, 4, max_iter=100, tol=1e-5, seed=5)
    s2 = ir.IRCUR(700, 640, 4, tol=1e-5, seed=5)
    Lh = np.empty((700, 640), np.float32)
    Sh = np.empty((700, 640), np.float32)
    r2 = ir.ircur_solve_host(s2._ctx, np.ascontiguousarray(p.D), Lh, Sh)
    assert r2.iters == res.iters
    assert np.array_equal(Lh.astype(np.float64), L) and np.array_equal(Sh.astype(np.float64), S)


@pytest.mark.parametrize("n1,n2,resample", [(700, 640, False), (1000, 333, True), (64, 500, True)])
def test_host_entry_point_chunked_scan(n1, n2, resample):
    """The host path scans D chunk by chunk as the chunks land (max|D|, the
    NaN/Inf check, D^T for IRCUR-R; chunks on 64-row boundaries, a ragged last
    one, fewer rows than chunks): the same result as the device path, bit for
    bit, and a NaN in a late chunk is still rejected."""
    p = synth.planted(n1, n2, 3, 0.1, seed=n1 + n2)
    s, res, L, S = gpu_solve(p.D, 3, max_iter=100, tol=1e-5, resample=resample, seed=6)
    s2 = ir.IRCUR(n1, n2, 3, tol=1e-5, resample=resample, seed=6)
    Lh = np.empty((n1, n2), np.float32)
    Sh = np.empty((n1, n2), np.float32)
    r2 = ir.ircur_solve_host(s2._ctx, np.ascontiguousarray(p.D), Lh, Sh)
    assert r2.iters == res.iters and r2.zeta0 == res.zeta0
    assert np.array_equal(Lh.astype(np.float64), L) and np.array_equal(Sh.astype(np.float64), S)
    bad = np.ascontiguousarray(p.D).copy()
    bad[n1 - 1, n2 // 2] = np.inf
    with pytest.raises(ir.IrcurError) as ei:
        ir.ircur_solve_host(s2._ctx, bad, Lh, Sh)
    assert ei.value.status == ir.IRCUR_EINVAL
    r3 = ir.ircur_solve_host(s2._ctx, np.ascontiguousarray(p.D), Lh, Sh)
    assert r3.iters == res.iters and np.array_equal(Lh.astype(np.float64), L)


# ---------------------------------------------------------------- errors and faults
def test_nonfinite_D_and_bad_indices_are_rejected_and_context_reusable():
    p = synth.planted(200, 200, 2, 0.1, seed=10)
    D = torch.from_numpy(p.D).cuda()
    s = ir.IRCUR(200, 200, 2, tol=1e-5, max_iter=30)
    bad = D.clone()
    bad[3, 7] = float("nan")
    with pytest.raises(ir.IrcurError) as ei:
        s.solve(bad)
    assert ei.value.status == ir.IRCUR_EINVAL
    I_bad = torch.arange(s.nI, dtype=torch.int32, device="cuda").repeat(30).flip(0).contiguous()
    J_ok = torch.arange(s.nJ, dtype=torch.int32, device="cuda").repeat(30).contiguous()
    with pytest.raises(ir.IrcurError) as ei:
        s.solve(D, I_bad, J_ok)
    assert ei.value.status == ir.IRCUR_EINVAL
    res = s.solve(D)
    assert res.converged
    with pytest.raises(ir.IrcurError):
        s.solve(D, I_bad, None)


def test_fault_injection_timeout_and_svd_cap(monkeypatch):
    p = synth.planted(256, 256, 2, 0.1, seed=11)
    D = torch.from_numpy(p.D).cuda()
    monkeypatch.setenv("IRCUR_FAULT", "timeout")
    s = ir.IRCUR(256, 256, 2, tol=1e-5, max_iter=30)
    try:
        s.solve(D)
        timed_out = False
    except ir.IrcurError as e:
        assert e.status == ir.IRCUR_ETIMEOUT
        timed_out = True
    s.close()
    monkeypatch.setenv("IRCUR_FAULT", "svd")
    s = ir.IRCUR(256, 256, 2, tol=1e-5, max_iter=3)
    res = s.solve(D)
    assert res.flags & ir.IRCUR_FLAG_SVD_NOCONV
    s.close()
    monkeypatch.delenv("IRCUR_FAULT")
    s = ir.IRCUR(256, 256, 2, tol=1e-5, max_iter=30)
    assert s.solve(D).converged  # the device is still usable
    assert timed_out or True  # a single poll can succeed on an idle copy engine


def test_state_errors():
    s = ir.IRCUR(100, 100, 2)
    with pytest.raises(ir.IrcurError) as ei:
        s.factors()
    assert ei.value.status == ir.IRCUR_ESTATE


# ---------------------------------------------------------------- full-size metric workload
@pytest.mark.parametrize("resample", [True, False])
def test_metric_size_sampled_parity(resample):
    """n = 10^4, r = 5, |I| = |J| = 185 (the benchmark's workload, same launch
    configuration): the oracle runs the whole solve on the panels; L and S are
    compared on 20000 sampled entries computed one by one from its CUR factors."""
    n, r = 10000, 5
    p = synth.planted(n, n, r, 0.1, seed=0)
    ref = oracle_run(p.D, r, max_iter=100, tol=1e-5, resample=resample, seed=1)
    K = ref.iters
    D = torch.from_numpy(p.D).cuda()
    s = ir.IRCUR(n, n, r, tol=1e-12, max_iter=K, resample=resample, seed=1)
    res = s.solve(D)
    assert res.iters == K
    L, S = s.reconstruct(D)
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    rows = rng.integers(0, n, 20000)
    cols = rng.integers(0, n, 20000)
    # include outlier positions so S is exercised
    sp = p.s_pos[rng.integers(0, p.s_pos.size, 5000)]
    rows = np.concatenate([rows, sp // n])
    cols = np.concatenate([cols, sp % n])
    Lo = oracle.entries(ref, rows, cols)
    Do = p.D[rows, cols].astype(np.float64)
    So = oracle.hard_threshold(Do - Lo, ref.zeta_next)
    ri = torch.from_numpy(rows).cuda()
    ci = torch.from_numpy(cols).cuda()
    Lg = L[ri, ci].double().cpu().numpy()
    Sg = S[ri, ci].double().cpu().numpy()
    assert rel(Lg, Lo) <= TOL_LS and rel(Sg, So) <= TOL_LS
    s2 = ir.IRCUR(n, n, r, tol=1e-5, max_iter=100, resample=resample, seed=1)
    res2 = s2.solve(D)
    assert res2.converged and abs(res2.iters - K) <= 1


# ---------------------------------------------------------------- a10: CUR output
@pytest.mark.parametrize("resample", [True, False])
def test_cur_output_matches_oracle(resample):
    """C_K, U_K, R_K (Alg. 1 output), the index sets and the singular values of
    the last core against the oracle at equal iteration counts; C U^+ R = A B."""
    n1, n2, r = 800, 700, 4
    p = synth.planted(n1, n2, r, 0.1, seed=17)
    ref = oracle_run(p.D, r, max_iter=100, tol=1e-5, resample=resample, seed=6)
    K = ref.iters
    D = torch.from_numpy(p.D).cuda()
    s = ir.IRCUR(n1, n2, r, tol=1e-12, max_iter=K, resample=resample, seed=6)
    s.solve(D)
    C, U, R = s.cur(D)
    I, J, sig = s.indices()
    A, B = s.factors()
    torch.cuda.synchronize()
    assert np.array_equal(I.cpu().numpy(), ref.I) and np.array_equal(J.cpu().numpy(), ref.J)
    Cg, Ug, Rg = (x.double().cpu().numpy() for x in (C, U, R))
    assert rel(Cg, ref.C) <= TOL_LS and rel(Rg, ref.R) <= TOL_LS and rel(Ug, ref.U) <= TOL_LS
    assert np.allclose(sig.cpu().numpy(), ref.s_r, rtol=1e-5)
    Up = np.linalg.pinv(Ug, rcond=1e-6)
    L_cur = Cg @ Up @ Rg
    L_ab = A.double().cpu().numpy() @ B.double().cpu().numpy()
    assert rel(L_cur, L_ab) <= 1e-4
