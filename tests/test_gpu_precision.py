"""Precision variant (IRCUR_PRECISION_BF16_PANELS): BF16 compact panels with the
threshold decision re-taken in FP32 inside the BF16 rounding band.

Pins, independent of the variant's own arithmetic:
* on data whose every entry is exactly representable in BF16, storing the
  panels in BF16 loses nothing, so the variant must equal the FP32 path bit
  for bit over many iterations (catches any error in the BF16 gather, staging,
  layout or conversion);
* entries placed at zeta_0 (1 +- 2^-11) (FP32 values whose BF16 rounding lands
  on zeta_0, the wrong side of a strict >) must still be classified as the
  FP32 path classifies them: one iteration equals the FP32 path bit for bit;
* on non-representable data the error against the FP64 oracle is bounded by
  the BF16 rounding of the kept entries (relative 2^-9 ~ 2e-3 per entry; the
  rank-r projection averages it down, measured ~1.3e-4 on planted data), and
  the error against the planted/background truth equals the FP32 path's.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2010_07422_gb300 import ircur as ir  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402

BF16_REL = 2.0 ** -9


def to_bf16_representable(x):
    """Round FP32 values to the nearest BF16 value (ties to even), kept as FP32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def solve(D, r, precision, **kw):
    n1, n2 = D.shape
    s = ir.IRCUR(n1, n2, r, resample=False, precision=precision, **kw)
    Dt = torch.from_numpy(np.ascontiguousarray(D, np.float32)).cuda()
    res = s.solve(Dt)
    L, S = s.reconstruct(Dt)
    A, B = s.factors()
    torch.cuda.synchronize()
    out = (res, L.double().cpu().numpy(), S.double().cpu().numpy(), A.cpu().numpy(), B.cpu().numpy())
    s.close()
    return out


def test_bf16_representable_data_is_bit_exact():
    p = synth.planted(1000, 900, 5, 0.1, seed=0)
    D = to_bf16_representable(p.D)
    a = solve(D, 5, ir.IRCUR_PRECISION_FP32, tol=1e-12, max_iter=20, seed=1)
    b = solve(D, 5, ir.IRCUR_PRECISION_BF16_PANELS, tol=1e-12, max_iter=20, seed=1)
    assert a[0].iters == b[0].iters == 20
    assert a[0].final_err == b[0].final_err
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


def test_threshold_band_is_decided_in_fp32():
    p = synth.planted(800, 700, 4, 0.1, seed=3)
    D = to_bf16_representable(p.D).copy()
    z0 = 4.0
    rng = np.random.default_rng(3)
    flat = D.reshape(-1)
    idx = rng.choice(flat.size, 20000, replace=False)
    mag = np.where(rng.random(idx.size) < 0.5, 1 + 2.0 ** -11, 1 - 2.0 ** -11)
    sign = np.where(rng.random(idx.size) < 0.5, 1.0, -1.0)
    flat[idx] = (z0 * mag * sign).astype(np.float32)
    # their BF16 rounding is exactly zeta_0: a strict > on the BF16 value would keep them all
    assert np.all(np.abs(to_bf16_representable(flat[idx])) == z0)
    a = solve(D, 4, ir.IRCUR_PRECISION_FP32, tol=1e-12, max_iter=1, seed=2, zeta0=z0)
    b = solve(D, 4, ir.IRCUR_PRECISION_BF16_PANELS, tol=1e-12, max_iter=1, seed=2, zeta0=z0)
    assert np.array_equal(a[3], b[3]) and np.array_equal(a[4], b[4])


@pytest.mark.parametrize("n,r,alpha", [(1000, 5, 0.1), (2500, 5, 0.2)])
def test_planted_error_against_oracle(n, r, alpha):
    p = synth.planted(n, n, r, alpha, seed=2)
    ref = oracle.ircur(p.D, r, 0.0, 0.7, 1e-5, 100, seed=1)
    Lo, So = oracle.dense_outputs(p.D, ref)
    K = ref.iters
    a = solve(p.D, r, ir.IRCUR_PRECISION_FP32, tol=1e-12, max_iter=K, seed=1)
    b = solve(p.D, r, ir.IRCUR_PRECISION_BF16_PANELS, tol=1e-12, max_iter=K, seed=1)
    assert rel(a[1], Lo) <= 1e-5
    assert rel(b[1], Lo) <= BF16_REL, rel(b[1], Lo)
    assert rel(b[1], p.L_true()) <= BF16_REL
    # the stopping value has a floor of the order of the BF16 rounding
    assert b[0].final_err <= BF16_REL


def test_video_shaped_equal_accuracy_against_background():
    """19200 x 3055 (120 x 160 pixels x frames), rank 2, 30 iterations."""
    v = synth.video_like(120, 160, 3055, seed=5)
    ref = oracle.ircur(v.D, 2, 0.0, 0.7, 1e-12, 30, seed=1)
    Lo, _ = oracle.dense_outputs(v.D, ref, with_sparse=False)
    a = solve(v.D, 2, ir.IRCUR_PRECISION_FP32, tol=1e-12, max_iter=30, seed=1)
    b = solve(v.D, 2, ir.IRCUR_PRECISION_BF16_PANELS, tol=1e-12, max_iter=30, seed=1)
    assert rel(b[1], Lo) <= BF16_REL, rel(b[1], Lo)
    ea, eb = rel(a[1], v.background), rel(b[1], v.background)
    assert abs(eb - ea) <= 0.05 * ea, (ea, eb)


def test_precision_variant_errors():
    lib = ir._lib()
    import ctypes
    P = ir.ircur_params
    ctx = ctypes.c_void_p()
    q = P(n1=300, n2=300, r=2, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=10, resample=1, seed=0,
          precision=ir.IRCUR_PRECISION_BF16_PANELS, svd_form=0)
    assert lib.ircur_create(ctypes.byref(q), None, ctypes.byref(ctx)) == ir.IRCUR_ENOTSUP
    q.precision = 2
    q.resample = 0
    assert lib.ircur_create(ctypes.byref(q), None, ctypes.byref(ctx)) == ir.IRCUR_ENOTSUP
    q.precision = ir.IRCUR_PRECISION_BF16_PANELS
    b = ctypes.c_void_p()
    assert lib.ircur_batch_create((P * 1)(q), 1, None, ctypes.byref(b)) == ir.IRCUR_ENOTSUP
    s = ir.IRCUR(300, 300, 2, resample=False, precision=ir.IRCUR_PRECISION_BF16_PANELS)
    with pytest.raises(ir.IrcurError) as e:
        s.record(True)
    assert e.value.status == ir.IRCUR_ENOTSUP
    s.close()
