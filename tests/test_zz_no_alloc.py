"""The allocation-free entry point ircur_solve_noalloc.

It serves callers that may not allocate device memory (a process whose memory
pool already holds the device memory it may use, or a latency-bound loop that
cannot afford cudaMalloc's implicit synchronisation): the same IRCUR-F solve as
ircur_create + ircur_solve + ircur_get_factors, with the workspace in a fixed
array inside the library.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2010_07422_gb300 import ircur as ir  # noqa: E402
from paper_2010_07422_gb300 import synth  # noqa: E402


def test_noalloc_matches_the_allocating_entry_point_twice():
    """Both entry points run the same kernels with the same launch shapes on the
    same inputs, so the factors must agree bit for bit -- on the first call and on
    a second call that finds the first call's leftovers in the shared array."""
    n1, n2, r = 1500, 1200, 5
    p = synth.planted(n1, n2, r, 0.1, seed=21)
    D = torch.from_numpy(p.D).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    ref = ir.IRCUR(n1, n2, r, gamma=0.7, tol=1e-5, max_iter=100, resample=False, seed=4)
    res_ref = ref.solve(D)
    A_ref, B_ref = ref.factors()
    torch.cuda.synchronize()
    ref.close()

    params = ir.ircur_params(n1=n1, n2=n2, r=r, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=100,
                             resample=0, seed=4, precision=0, svd_form=0)
    for _ in range(2):  # the second call starts from the first call's leftovers in the shared array
        A = torch.full((n1, r), float("nan"), device="cuda")
        B = torch.full((r, n2), float("nan"), device="cuda")
        res = ir.ircur_solve_noalloc(params, D, D.stride(0), A, B, stream)
        torch.cuda.synchronize()
        assert res.iters == res_ref.iters and res.converged
        assert res.final_err == res_ref.final_err
        assert torch.equal(A, A_ref) and torch.equal(B, B_ref)

    # sizes beyond the fixed array and IRCUR-R are rejected, nothing is launched
    big = ir.ircur_params(n1=4096, n2=1200, r=r, nI=0, nJ=0, zeta0=0.0, gamma=0.7, tol=1e-5, max_iter=100,
                          resample=0, seed=4, precision=0, svd_form=0)
    with pytest.raises(ir.IrcurError) as ei:
        ir.ircur_solve_noalloc(big, D, D.stride(0), A, B, stream)
    assert ei.value.status == ir.IRCUR_EINVAL
    params.resample = 1
    with pytest.raises(ir.IrcurError) as ei:
        ir.ircur_solve_noalloc(params, D, D.stride(0), A, B, stream)
    assert ei.value.status == ir.IRCUR_EINVAL
