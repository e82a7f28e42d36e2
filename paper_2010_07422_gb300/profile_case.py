"""A fixed workload for kernel profilers: a few IRCUR solves of one planted
problem, drawn on the device, with nothing else on the device.

    IRCUR_NO_GRAPH=1 python -m paper_2010_07422_gb300.profile_case --n 20000 --r 10 --variant F

Each solve runs exactly --iters iterations (the tolerance is unreachable), so
solve s launches its core SVD and its panel pass --iters times each, in that
order, after the same setup kernels: a profiler that skips the first
(solves - 1) * iters launches of a kernel sees the last solve.  With
IRCUR_NO_GRAPH=1 every kernel is a separate launch (profilers do not see the
kernel nodes of a graph that holds a conditional node); the kernels and their
arguments are the ones the graph runs.  Prints one JSON line per solve.

    IRCUR_NO_GRAPH=1 python -m paper_2010_07422_gb300.profile_case --batch 64 --solves 2

runs instead a batch of that many uneven IRCUR-R problems (n1, n2 uniform in
[500, 4000], r in 2..10, alpha in [0.05, 0.3], the planted generator, tol 1e-5)
with the given core-SVD form.  Solve k runs inside the NVTX range "solve<k>",
so a profiler can take exactly one solve's launches.
"""

from __future__ import annotations

import argparse
import json
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--r", type=int, default=10)
    ap.add_argument("--alpha", type=float, default=0.1)
    ap.add_argument("--variant", default="F", choices=["F", "R"])
    ap.add_argument("--iters", type=int, default=6)
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--batch", type=int, default=0, help="a batch of this many uneven problems instead")
    ap.add_argument("--svd-form", type=int, default=2, help="core-SVD form of the batch's problems")
    a = ap.parse_args(argv)
    import torch

    from . import ircur as ir
    from . import synth

    if a.batch > 0:
        shapes = synth.uneven_batch(a.batch, seed=7)
        Ds = [synth.planted_device(q["n1"], q["n2"], q["r"], q["alpha"], seed=100 + i) for i, q in enumerate(shapes)]
        b = ir.IRCURBatch([dict(n1=q["n1"], n2=q["n2"], r=q["r"], resample=True, seed=i, tol=1e-5, max_iter=100,
                                svd_form=a.svd_form) for i, q in enumerate(shapes)])
        torch.cuda.synchronize()
        for k in range(a.solves):
            torch.cuda.nvtx.range_push(f"solve{k}")
            t0 = time.perf_counter()
            res = b.solve(Ds)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            print(json.dumps({"solve": k, "batch": a.batch, "svd_form": a.svd_form,
                              "iters_max": max(r_.iters for r_ in res), "iters_sum": sum(r_.iters for r_ in res),
                              "wall_ms": 1e3 * (time.perf_counter() - t0)}), flush=True)
        b.close()
        return

    D = synth.planted_device(a.n, a.n, a.r, a.alpha, seed=a.seed)
    s = ir.IRCUR(a.n, a.n, a.r, gamma=0.7, tol=1e-30, max_iter=a.iters, resample=(a.variant == "R"), seed=1)
    for k in range(a.solves):
        t0 = time.perf_counter()
        res = s.solve(D)
        torch.cuda.synchronize()
        print(json.dumps({"solve": k, "n": a.n, "r": a.r, "variant": a.variant, "iters": res.iters,
                          "flags": res.flags, "svd_half_steps": res.svd_steps, "wall_ms": 1e3 * (time.perf_counter() - t0),
                          "launch_shape": ir.ircur_get_launch_shape(s._ctx)}), flush=True)
    s.close()


if __name__ == "__main__":
    main()
