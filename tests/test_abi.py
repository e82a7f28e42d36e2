"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/ircur.h declares; the Python binding wraps each one."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ircur_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2010_07422_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("ircur_create", "ircur_solve", "ircur_reconstruct", "ircur_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2010_07422_gb300 import ircur
    assert set(declared_functions()) <= set(ircur.EXPORTED)


def test_status_strings_and_param_validation_without_gpu(lib):
    """Argument checks run on the host before any CUDA call."""
    from paper_2010_07422_gb300 import ircur as ir
    lib = ir._lib()
    assert lib.ircur_status_string(ir.IRCUR_EINVAL).decode().startswith("IRCUR_EINVAL")
    ctx = ctypes.c_void_p()

    def create(**kw):
        base = dict(n1=100, n2=80, r=3, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=10,
                    resample=1, seed=0, precision=0, svd_form=0)
        base.update(kw)
        return lib.ircur_create(ctypes.byref(ir.ircur_params(**base)), None, ctypes.byref(ctx))

    assert create(r=0) == ir.IRCUR_EINVAL
    assert create(r=21) == ir.IRCUR_ENOTSUP
    assert create(gamma=1.0) == ir.IRCUR_EINVAL
    assert create(gamma=0.0) == ir.IRCUR_EINVAL
    assert create(tol=0.0) == ir.IRCUR_EINVAL
    assert create(max_iter=0) == ir.IRCUR_EINVAL
    assert create(nI=2) == ir.IRCUR_EINVAL        # |I| < r violates Thm 1's |I| >= r
    assert create(nJ=81) == ir.IRCUR_EINVAL       # |J| > n2
    assert create(resample=2) == ir.IRCUR_EINVAL
    assert create(precision=1) == ir.IRCUR_ENOTSUP
    assert create(svd_form=3) == ir.IRCUR_EINVAL
    assert create(svd_form=-1) == ir.IRCUR_EINVAL
    assert create(n1=0) == ir.IRCUR_EINVAL
    assert ctx.value is None
    # batch argument checks (before any CUDA call)
    good = ir.ircur_params(n1=100, n2=80, r=3, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=10,
                           resample=1, seed=0, precision=0, svd_form=0)
    bad = ir.ircur_params(n1=100, n2=80, r=3, nI=0, nJ=0, zeta0=0.0, gamma=1.5, tol=1e-5, max_iter=10,
                          resample=1, seed=0, precision=0, svd_form=0)
    bh = ctypes.c_void_p()
    assert lib.ircur_batch_create((ir.ircur_params * 1)(good), 0, None, ctypes.byref(bh)) == ir.IRCUR_EINVAL
    assert lib.ircur_batch_create((ir.ircur_params * 2)(good, bad), 2, None, ctypes.byref(bh)) == ir.IRCUR_EINVAL
    assert lib.ircur_batch_create(None, 1, None, ctypes.byref(bh)) == ir.IRCUR_EINVAL
    assert bh.value is None
    assert lib.ircur_batch_instance(None, 0) is None
    # streaming argument checks
    assert lib.ircur_stream_columns(None, None, 0, 1, 0, None, 0, None, 0) == ir.IRCUR_EINVAL
    # launch-shape query
    assert lib.ircur_get_launch_shape(None, None, None, None) == ir.IRCUR_EINVAL
    # adjoint argument checks
    assert lib.ircur_set_record(None, 1) == ir.IRCUR_EINVAL
    assert lib.ircur_backward(None, None, 0, None, 0, None, 0, None, 0) == ir.IRCUR_EINVAL
    # sampler argument checks
    assert lib.ircur_sample_indices(0, 0, 0, 10, 11, None, None) == ir.IRCUR_EINVAL
    assert lib.ircur_sample_indices(0, 0, 2, 10, 5, ctypes.c_void_p(16), None) == ir.IRCUR_EINVAL


def test_fault_injection_alloc_returns_enomem(lib, monkeypatch):
    from paper_2010_07422_gb300 import ircur as ir
    monkeypatch.setenv("IRCUR_FAULT", "alloc")
    ctx = ctypes.c_void_p()
    p = ir.ircur_params(n1=100, n2=80, r=3, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=10,
                        resample=1, seed=0, precision=0, svd_form=0)
    assert ir._lib().ircur_create(ctypes.byref(p), None, ctypes.byref(ctx)) == ir.IRCUR_ENOMEM
    assert ctx.value is None
    bh = ctypes.c_void_p()
    assert ir._lib().ircur_batch_create((ir.ircur_params * 2)(p, p), 2, None, ctypes.byref(bh)) == ir.IRCUR_ENOMEM
    assert bh.value is None


def declared_arity():
    """Parameter count of every function include/ircur.h declares."""
    out = {}
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(ircur_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", text):
            args = m.group(2).strip()
            out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(lib):
    """The ctypes argtypes of every entry point have as many arguments as its
    declaration (an ABI change in one place and not the other fails here)."""
    from paper_2010_07422_gb300 import ircur
    lib_bound = ircur._lib()
    arity = declared_arity()
    assert set(arity) == set(declared_functions())
    for name, n in arity.items():
        argtypes = getattr(lib_bound, name).argtypes
        if argtypes is None:  # no-argument functions are left without argtypes
            assert n == 0, name
            continue
        assert len(argtypes) == n, (name, len(argtypes), n)
