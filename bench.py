#!/usr/bin/env python
"""IRCUR benchmark: time-to-tolerance and iterations/s at n1 = n2 = 10^4, r = 5.

One step = one whole pass of the hot path on one synthetic D: index sampling,
zeta_0 = max|D|, the iterations of Alg. 1 until e_k <= 1e-5 (IRCUR-R: fresh
I, J every iteration), then the dense L = C U^+ R and S = T_zeta(D - L).
D (400 MB FP32) is larger than L2, so every step starts cold.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun every rank solves its own independent instance (different
seed): the method has no exchange between independent problems, so N GPUs run
N replicas (weak scaling) with no data-path collective; rank 0 prints one JSON
line with the whole-job iterations/s (sum over ranks / max time over ranks).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IRCUR time-to-1e-5 rel err & iters/s at n=10^4,r=5; HBM GB/s % of peak"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default="R", choices=["R", "F"])
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--r", type=int, default=5)
    ap.add_argument("--alpha", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the headline line: one JSON line per configuration of the size sweep "
                         "(n in 1000, 2500, 5000, 10000, 20000; r in 5, 10; alpha in 0.1, 0.2, 0.3; F and R)")
    ap.add_argument("--phase-transition", action="store_true",
                    help="instead of the headline line: recovery rates over (c_I, alpha) at n = 1000 "
                         "(50 trials per cell, r = 5, 10 and 20, IRCUR-F and -R) on the batched solver")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default pass launch shape (fixed launch sequence, for profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary measurements (batched, adjoint, precision variant)")
    return ap.parse_args()


def workload_name(a):
    nI = math.ceil(4 * a.r * math.log(a.n))
    return (f"IRCUR-{a.variant} planted rank-{a.r} + {a.alpha:g}-sparse D, n1=n2={a.n}, |I|=|J|={nI}, "
            f"zeta0=max|D|, gamma=0.7, tol=1e-5, max_iter=100, then dense L and S")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dram_traffic(kernel, workload_tag):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
    an ncu capture recorded in profiles/dram_traffic.json, or None when no
    capture exists or the kernel's source file changed since it was taken."""
    prof = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(prof) as f:
            caps = json.load(f)["captures"]
    except Exception:
        return None
    for c in caps:
        if c.get("kernel") != kernel or c.get("workload") != workload_tag:
            continue
        src = os.path.join(ROOT, "paper_2010_07422_gb300", "csrc", c["source"])
        if not os.path.exists(src):
            return None
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:12]
        return float(c["bytes"]) if sha == c["sha256_12"] else None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms in the background,
    each sample stamped with the host clock when it is read."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, t0=None, t1=None):
        """Statistics of the samples read between host times t0 and t1 (the timed
        region, widened by one sampling period each side); of every sample since
        start() (warm-up and timed region) if none fell inside."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        window = "warm-up and timed region"
        if t0 is not None:
            inside = [x for x in self.lines if t0 - 0.05 <= x[0] <= t1 + 0.05]
            if inside:
                lines, window = inside, "timed region"
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names[1:], parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def rank_seed(seed, rank):
    """Each rank solves its own independent instance (weak scaling, no exchange)."""
    return seed + 1000 * rank


def make_input(a, rank):
    from paper_2010_07422_gb300 import synth
    return synth.planted(a.n, a.n, a.r, a.alpha, seed=rank_seed(a.seed, rank))


def aggregate(dist, world, elapsed, units, device):
    """Whole-job figures over the ranks: the slowest rank's elapsed time and the
    units every rank processed (one all-reduce each; no data-path collective)."""
    if world <= 1:
        return float(elapsed), float(units)
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cpu_oracle_sample(p, a, seconds, max_steps=None):
    """The FP64 oracle as it stands, timed on the host cores: whole IRCUR solves
    (same workload, same variant) until about `seconds` of CPU work."""
    import oracle
    D64 = p.D  # the oracle promotes to FP64 per panel gather
    t0 = time.perf_counter()
    iters = solves = 0
    last = None
    while True:
        res = oracle.ircur(D64, a.r, 0, 0.7, 1e-5, 100, resample=(a.variant == "R"), seed=a.seed + 1 + solves)
        iters += res.iters
        solves += 1
        last = res
        el = time.perf_counter() - t0
        if el >= seconds or (max_steps and solves >= max_steps):
            break
    return iters, solves, el, last


def run_reference(a, rank, world):
    """--impl reference: the FP64 CPU oracle on the same workload, rank 0 only.
    Each step is a bounded sample: an oracle solve truncated to a fixed number
    of iterations chosen so that warmup + steps end within about two minutes."""
    if rank != 0:
        return
    import oracle
    p = make_input(a, 0)
    # calibrate one iteration
    t0 = time.perf_counter()
    oracle.ircur(p.D, a.r, 0, 0.7, 1e-5, 1, resample=(a.variant == "R"), seed=a.seed + 1)
    t_it = time.perf_counter() - t0
    per_step = int(max(1, min(100, 110.0 / max(1e-3, t_it) / max(1, a.steps + a.warmup))))
    for w in range(a.warmup):
        oracle.ircur(p.D, a.r, 0, 0.7, 1e-5, per_step, resample=(a.variant == "R"), seed=a.seed + 1 + w)
    t0 = time.perf_counter()
    iters = 0
    for s in range(a.steps):
        res = oracle.ircur(p.D, a.r, 0, 0.7, 1e-5, per_step, resample=(a.variant == "R"), seed=a.seed + 1 + s)
        iters += res.iters
    el = time.perf_counter() - t0
    value = iters / el
    cores = os.cpu_count()
    sample = (f"{a.steps} steps x oracle solve truncated to {per_step} iterations "
              f"(numpy FP64, n={a.n}, r={a.r}, IRCUR-{a.variant})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * el / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "n1": a.n, "n2": a.n, "r": a.r, "alpha": a.alpha,
                       "variant": a.variant, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _timed(fn, reps, stream):
    """Median of `reps` CUDA-event timings (ms) of fn() on `stream`."""
    import torch
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def bench_batched(ir, synth, stream, count=64, seed=7):
    """Uneven independent problems (n1, n2 uniform in [500, 4000], r in 2..10,
    alpha in [0.05, 0.3], the planted generator): one batch with each of the
    three core-SVD forms (one CTA, clusters of 16, clusters of 8), the fastest
    reported, vs a loop of single solves (default form) on the same GPU.
    Solves/s."""
    import torch
    shapes = synth.uneven_batch(count, seed=seed)
    Ds = [synth.planted_device(q["n1"], q["n2"], q["r"], q["alpha"], seed=100 + i) for i, q in enumerate(shapes)]
    probs = [dict(n1=q["n1"], n2=q["n2"], r=q["r"], resample=True, seed=i, tol=1e-5, max_iter=100)
             for i, q in enumerate(shapes)]
    batch_cl = ir.IRCURBatch(probs)
    for _ in range(2):
        batch_cl.solve(Ds)
    batch_cl.autotune(Ds, reps=3)
    t_batch_cl = _timed(lambda: batch_cl.solve(Ds), 5, stream)
    batch_cl.close()
    batch_c8 = ir.IRCURBatch([dict(q, svd_form=ir.IRCUR_SVD_CLUSTER8) for q in probs])
    for _ in range(2):
        batch_c8.solve(Ds)
    batch_c8.autotune(Ds, reps=3)
    t_batch_c8 = _timed(lambda: batch_c8.solve(Ds), 5, stream)
    batch_c8.close()
    batch = ir.IRCURBatch([dict(q, svd_form=ir.IRCUR_SVD_ONE_CTA) for q in probs])
    for _ in range(2):
        res = batch.solve(Ds)
    tune = batch.autotune(Ds, reps=3)
    for _ in range(2):
        res = batch.solve(Ds)
    t_batch = _timed(lambda: batch.solve(Ds), 5, stream)
    singles = [ir.IRCUR(q["n1"], q["n2"], q["r"], resample=True, seed=q["seed"], tol=1e-5, max_iter=100)
               for q in probs]
    for s_, D_ in zip(singles, Ds):
        s_.solve(D_)
    t_loop = _timed(lambda: [s_.solve(D_) for s_, D_ in zip(singles, Ds)], 3, stream)
    iters = [r_.iters for r_ in res]
    forms = {"one CTA where the core fits (svd_form 1)": t_batch,
             "cluster of 16 CTAs (svd_form 0, the lone-solve default)": t_batch_cl,
             "cluster of 8 CTAs (svd_form 2)": t_batch_c8}
    best = min(forms, key=lambda k_: forms[k_])
    t_best = forms[best]
    out = {"workload": f"{count} independent IRCUR-R problems, n1, n2 uniform in [500, 4000], r uniform in 2..10, "
                       "alpha uniform in [0.05, 0.3], planted generator on the device, tol 1e-5",
           "solves_per_s": count / (t_best / 1e3), "ms_per_batch": t_best,
           "svd_form": best + ", the fastest of the three timed",
           "one_cta_form_solves_per_s": count / (t_batch / 1e3),
           "cluster_form_solves_per_s": count / (t_batch_cl / 1e3),
           "cluster8_form_solves_per_s": count / (t_batch_c8 / 1e3),
           "loop_solves_per_s": count / (t_loop / 1e3), "loop_ms": t_loop, "speedup_vs_loop": t_loop / t_best,
           "iters_min_max": [min(iters), max(iters)], "converged": int(sum(r_.converged for r_ in res)),
           "autotune": tune}
    for s_ in singles:
        s_.close()
    batch.close()
    return out


def bench_adjoint(ir, synth, stream, count=8, n=4096, r=10, T=15):
    """Unrolled IRCUR-F forward + hand-written backward through autograd:
    loss = ||L - L_true||_F^2 + 0.1 ||S||_1 per instance."""
    import torch
    gens = [synth.planted_device(n, n, r, 0.1, seed=300 + b) for b in range(count)]
    solvers = [ir.IRCUR(n, n, r, tol=1e-12, max_iter=T, resample=False, seed=b) for b in range(count)]
    Lt = torch.zeros(n, n, device="cuda")

    def step():
        for D0, s_ in zip(gens, solvers):
            D = D0.detach().requires_grad_(True)
            L, S = ir.ircur_unrolled(D, s_)
            loss = ((L - Lt) ** 2).sum() + 0.1 * S.abs().sum()
            loss.backward()

    for _ in range(2):
        step()
    t = _timed(step, 5, stream)
    dL = torch.randn(n, n, device="cuda")
    tf = _timed(lambda: (solvers[0].solve(gens[0]), solvers[0].reconstruct(gens[0])), 5, stream)
    tb = _timed(lambda: solvers[0].backward(gens[0], dL, dL), 5, stream)
    for s_ in solvers:
        s_.close()
    return {"workload": f"{count} instances n1 = n2 = {n}, r = {r}, alpha = 0.1, fixed I, J "
                        f"(|I| = |J| = {ir.sample_size(4, r, n)}), T = {T} unrolled iterations; "
                        "loss ||L - L_true||^2 + 0.1 ||S||_1 through torch.autograd",
            "fwd_bwd_ms": t, "per_instance_forward_ms": tf, "per_instance_backward_ms": tb,
            "note": "gradient parity with the FP64 oracle gradient: tests/test_gpu_adjoint.py"}


def bench_stream(ir, synth, stream, n=10000, c=1024, r=5):
    """New columns against a solved model: planted D of n x (n + c) drawn on
    the device, IRCUR-F solve on the first n columns, the last c streamed
    (ircur_stream_columns, the solve's iteration count).  Columns/s, and the
    dense part's HBM rate (read the new columns, write L and S)."""
    import torch
    Dall = synth.planted_device(n, n + c, r, 0.1, seed=41)
    D = Dall[:, :n].contiguous()
    Dn = Dall[:, n:].contiguous()
    del Dall
    s_ = ir.IRCUR(n, n, r, tol=1e-5, max_iter=100, resample=False, seed=3)
    res = s_.solve(D)
    for _ in range(3):
        s_.stream_columns(Dn)
    t = _timed(lambda: s_.stream_columns(Dn), 20, stream)
    out = {"workload": f"planted n1 = {n}, model solved on {n} columns (IRCUR-F, r = {r}, alpha = 0.1), "
                       f"{c} new columns streamed with {res.iters} iterations each",
           "columns_per_s": c / (t / 1e3), "ms_per_call": t,
           "dense_gbs": 12.0 * n * c / (t * 1e-3) / 1e9}
    s_.close()
    return out


def bench_precision(ir, synth, stream, K=30):
    """Video-shaped D (120 x 160 pixels x 3055 frames, r = 2): FP32 panels vs
    BF16 panels with the FP32 band re-check, same K iterations."""
    import torch
    v = synth.video_like(120, 160, 3055, seed=5)
    D = torch.from_numpy(v.D).cuda()
    out = {"workload": "video-shaped D 19200 x 3055 (120 x 160 pixels x frames), r = 2, IRCUR-F, "
                       f"{K} iterations, values in [0, 1]"}
    Ls = {}
    for name, prec in (("fp32", ir.IRCUR_PRECISION_FP32), ("bf16_panels", ir.IRCUR_PRECISION_BF16_PANELS)):
        s_ = ir.IRCUR(19200, 3055, 2, resample=False, precision=prec, tol=1e-12, max_iter=K, seed=1)
        for _ in range(3):
            s_.solve(D)
        out[name + "_solve_ms"] = _timed(lambda: s_.solve(D), 10, stream)
        L, _ = s_.reconstruct(D, with_sparse=False)
        Ls[name] = L.double().cpu().numpy()
        out[name + "_rel_err_vs_background"] = float(np.linalg.norm(Ls[name] - v.background) /
                                                     np.linalg.norm(v.background))
        s_.close()
    out["bf16_rel_diff_vs_fp32_L"] = float(np.linalg.norm(Ls["bf16_panels"] - Ls["fp32"]) / np.linalg.norm(Ls["fp32"]))
    out["speedup_bf16_vs_fp32"] = out["fp32_solve_ms"] / out["bf16_panels_solve_ms"]
    out["note"] = "error against the FP64 oracle: tests/test_gpu_precision.py"
    return out


def run_sweep(a):
    """Time-to-tolerance over the size sweep (planted inputs drawn on the device;
    the FP64 oracle timed on the host for the sizes it finishes in seconds)."""
    import torch
    from paper_2010_07422_gb300 import ircur as ir
    from paper_2010_07422_gb300 import synth
    import oracle
    stream = torch.cuda.current_stream()
    for n in (1000, 2500, 5000, 10000, 20000):
        for r in (5, 10):
            for alpha in (0.1, 0.2, 0.3):
                if n == 1000 and (r, alpha) != (5, 0.1):
                    continue
                D = synth.planted_device(n, n, r, alpha, seed=n + r)
                for variant in ("F", "R"):
                    s_ = ir.IRCUR(n, n, r, tol=1e-5, max_iter=100, resample=(variant == "R"), seed=1)
                    s_.solve(D)
                    s_.autotune(D, reps=2)
                    res = s_.solve(D)
                    ms = _timed(lambda: s_.solve(D), 5, stream)
                    ir.ircur_set_trace(s_._ctx, True)
                    s_.solve(D)
                    spans = ir.ircur_get_trace(s_._ctx, 100)
                    pass_us = float(np.mean([q[2] for q in spans]))
                    pass_post_us = float(np.mean([q[3] for q in spans]))
                    svd_us = float(np.mean([q[1] for q in spans]))
                    nI, nJ, Rp = s_.nI, s_.nJ, (r if r <= 10 else 16)
                    pbytes = 4.0 * (nI + nJ) * n + 2 * 4.0 * Rp * 2 * n
                    pass_gbs = pbytes / (pass_us * 1e-6) / 1e9
                    L, _ = s_.reconstruct(D, with_sparse=False)
                    line = {"sweep": True, "n": n, "r": r, "alpha": alpha, "variant": variant, "m": nI,
                            "iters": res.iters, "converged": bool(res.converged), "time_to_tol_ms": ms,
                            "iters_per_s": res.iters / (ms / 1e3), "svd_us": svd_us,
                            "pass_us": pass_us, "pass_after_svd_us": pass_post_us,
                            "pass_bytes": pbytes, "pass_gbs": pass_gbs,
                            "pass_frac_of_measured_hbm": pass_gbs / peaks()[0],
                            "pass_gbs_after_svd": pbytes / (pass_post_us * 1e-6) / 1e9,
                            "span_note": "pass_us: first pass block start (it starts during the core SVD) to "
                                         "last block end; pass_after_svd_us: from its first return of the "
                                         "wait for the SVD"}
                    if n <= 2500:
                        Dn = D.cpu().numpy()
                        t0 = time.perf_counter()
                        ref = oracle.ircur(Dn, r, 0.0, 0.7, 1e-5, 100, resample=(variant == "R"), seed=1)
                        line["oracle_s"] = time.perf_counter() - t0
                        line["oracle_iters"] = ref.iters
                    s_.close()
                    print(json.dumps(line), flush=True)
                del D


def run_phase_transition(a, n=1000, trials=50, c_values=(0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0),
                         alphas=(0.05, 0.1, 0.15, 0.2, 0.25, 0.3, 0.35, 0.4, 0.45, 0.5)):
    """Empirical phase transition in (c_I, alpha) (Sec. 4.1, Fig. 1) on the
    batched solver: n = 1000, |I| = |J| = ceil(c_I r ln n), planted problems of
    the supplement's synthetic setup (outliers uniform in [-E|L|, E|L|],
    zeta_0 = 2 ||L||_inf, gamma = 0.65, stop at e_k <= 1e-5, at most 100
    iterations); success = ||L - L_true||_F / ||L_true||_F <= 1e-3.  One batch
    of len(alphas) x trials problems per (r, variant, c_I)."""
    import torch
    from paper_2010_07422_gb300 import ircur as ir
    from paper_2010_07422_gb300 import synth
    t_all = time.perf_counter()
    solves, t_solves = 0, 0.0
    for r in (5, 10, 20):
        for variant in ("F", "R"):
            for c_I in c_values:
                m = int(min(n, math.ceil(c_I * r * math.log(n))))
                probs, gens = [], []
                for ai, alpha in enumerate(alphas):
                    for tr in range(trials):
                        seed = 1_000_003 * r + 10_007 * ai + tr
                        D, W, V = synth.planted_device(n, n, r, alpha, seed=seed, outlier_scale=1.0,
                                                       return_factors=True)
                        z0 = 2.0 * float((W @ V.T).abs().max())
                        gens.append((D, W, V))
                        probs.append(dict(n1=n, n2=n, r=r, nI=m, nJ=m, resample=(variant == "R"), seed=seed,
                                          zeta0=z0, gamma=0.65, tol=1e-5, max_iter=100))
                try:
                    batch = ir.IRCURBatch(probs)
                except ir.IrcurError as e:
                    # the core (m x m at rank r) does not fit the GPU's shared memory
                    print(json.dumps({"phase_transition": True, "n": n, "r": r, "variant": variant, "c_I": c_I,
                                      "m": m, "unsupported": str(e)}), flush=True)
                    del gens
                    continue
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                batch.solve([g[0] for g in gens])
                torch.cuda.synchronize()
                t_solve = time.perf_counter() - t0
                t_solves += t_solve
                solves += len(probs)
                ok = []
                for i, (D, W, V) in enumerate(gens):
                    A, B = batch[i].factors()
                    Lt = W @ V.T
                    ok.append(float(torch.linalg.norm(A @ B - Lt) / torch.linalg.norm(Lt)) <= 1e-3)
                batch.close()
                rates = [sum(ok[ai * trials:(ai + 1) * trials]) / trials for ai in range(len(alphas))]
                print(json.dumps({"phase_transition": True, "n": n, "r": r, "variant": variant, "c_I": c_I,
                                  "m": m, "alphas": list(alphas), "success_rate": rates, "trials": trials,
                                  "batch_solve_s": round(t_solve, 4)}), flush=True)
                del gens
    print(json.dumps({"phase_transition_total_s": round(time.perf_counter() - t_all, 1), "solves": solves,
                      "batch_solve_total_s": round(t_solves, 3)}), flush=True)


def main():
    a = parse_args()
    if a.sweep:
        run_sweep(a)
        return
    if a.phase_transition:
        run_phase_transition(a)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_2010_07422_gb300 import ircur as ir

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    p = make_input(a, rank)
    n = a.n
    D = torch.from_numpy(p.D).cuda()
    L = torch.empty_like(D)
    S = torch.empty_like(D)
    resample = a.variant == "R"
    solver = ir.IRCUR(n, n, a.r, gamma=0.7, tol=1e-5, max_iter=100, resample=resample, seed=a.seed + 1 + rank)
    ir.ircur_set_trace(solver._ctx, True)  # per-kernel spans inside the graph (two atomics per block)
    stream = torch.cuda.current_stream()

    def step():
        res = solver.solve(D)
        solver.reconstruct(D, L=L, S=S)
        return res

    # clocks sampled from the warm-up on (nvidia-smi takes a while to report)
    clk = ClockSampler(local)
    clk.start()
    for _ in range(max(3, a.warmup)):
        step()
    # pass-kernel launch shape chosen by timing whole solves (ircur_autotune)
    tune = None
    if not a.no_autotune:
        tune = solver.autotune(D, reps=3)
        for _ in range(2):
            step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()

    t_host0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    rec = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    sol = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    iters = []
    flags = 0
    svd_steps = 0
    ev0.record(stream)
    for k in range(a.steps):
        sol[k][0].record(stream)
        res = solver.solve(D)
        sol[k][1].record(stream)
        rec[k][0].record(stream)
        solver.reconstruct(D, L=L, S=S)
        rec[k][1].record(stream)
        iters.append(res.iters)
        flags |= res.flags
        svd_steps += res.svd_steps
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop(t_host0, time.perf_counter())
    barrier()
    total_ms = ev0.elapsed_time(ev1)
    recon_ms = [s.elapsed_time(e) for s, e in rec]
    solve_ms = [s.elapsed_time(e) for s, e in sol]
    my_iters = float(sum(iters))
    total_ms_max, all_iters = aggregate(dist, world, total_ms, my_iters, "cuda")

    # accuracy of the last step against the planted truth, on sampled entries
    rng = np.random.default_rng(0)
    ri = rng.integers(0, n, 200000)
    ci = rng.integers(0, n, 200000)
    Lg = L[torch.from_numpy(ri).cuda(), torch.from_numpy(ci).cuda()].double().cpu().numpy()
    Lt = p.L_entries(ri, ci)
    rel_err_truth = float(np.linalg.norm(Lg - Lt) / np.linalg.norm(Lt))

    # Alg. 2 (CUR to SVD) of the last iterate, on request after the solve
    c2s_us = 1e3 * _timed(lambda: solver.svd(), 5, stream)

    # Per-kernel spans of the last timed step (device clock, inside the graph):
    # Phase I on the core (the SVD's prologue), the core SVD, the panel pass
    # from its first block's start (its blocks start while the SVD runs) and
    # from its first return of the wait for the SVD
    spans = ir.ircur_get_trace(solver._ctx, 100)
    K = len(spans)
    core_us = [q[0] for q in spans]
    svd_us = [q[1] for q in spans]
    pass_us = [q[2] for q in spans]
    pass_post_us = [q[3] for q in spans]
    rec_avg_us = float(np.mean(recon_ms)) * 1e3
    per_step_us = {"core_phase1_in_svd": float(np.sum(core_us)), "csvd_kernel": float(np.sum(svd_us)),
                   "pass_kernel": float(np.sum(pass_us)), "pass_kernel_after_svd": float(np.sum(pass_post_us)),
                   "recon_vec_kernel": rec_avg_us}
    hbm_peak, peak_src = peaks()
    peak_note = ("measured STREAM-style copy (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                 else "fallback 6.8 TB/s")
    nI, nJ, r = solver.nI, solver.nJ, a.r
    Rp = r if r <= 10 else (12 if r <= 12 else 16)

    def roof_hbm(kernel, bytes_per_launch, avg_us, tag):
        ach = bytes_per_launch / (avg_us * 1e-6) / 1e9
        return {"kernel": kernel, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": dram_traffic(kernel, tag), "peak_source": peak_note,
                "algorithmic_bytes_per_launch": bytes_per_launch, "avg_launch_us": avg_us}

    # reconstruction: read D, write L and S (12 bytes per entry) + the factors
    roof_recon = roof_hbm("recon_vec_kernel", 12.0 * n * n + 4.0 * r * 2 * n, rec_avg_us, f"n{n}_r{r}")
    # panel passes: the two panels once, A_k, B_k read, A_{k+1}, B_{k+1} written;
    # the full launch span (its tile loads overlap the SVD) sets the fraction,
    # the span after the SVD is the time it adds to an iteration
    pass_bytes = 4.0 * (nI * n + nJ * n) + 2 * 4.0 * Rp * (n + n)
    roof_pass = roof_hbm("pass_kernel", pass_bytes, float(np.mean(pass_us)), f"n{n}_r{r}")
    roof_pass["span"] = "first block start to last block end (its blocks start while the core SVD runs)"
    roof_pass["avg_after_svd_us"] = float(np.mean(pass_post_us))
    roof_pass["achieved_after_svd"] = pass_bytes / (roof_pass["avg_after_svd_us"] * 1e-6) / 1e9
    # core SVD: FP32 work per launch = one product of 2 nI nJ r flops per
    # half-step, plus its Cholesky QR (2 (nI or nJ) r^2), and Phase I on the core
    # (2 r flops per entry)
    hsteps = svd_steps / max(1.0, my_iters)
    svd_flops = hsteps * (2.0 * nI * nJ * r + (nI + nJ) * r * r) + 2.0 * r * nI * nJ
    fp32_peak = 152 * 128 * 2 * 2.070e9 / 1e12  # TFLOP/s: SMs x FP32 lanes x FMA x max SM clock
    svd_avg_us = float(np.mean(svd_us))
    svd_ach = svd_flops / (svd_avg_us * 1e-6) / 1e12
    nc_svd, pass_blocks, pass_bufs = ir.ircur_get_launch_shape(solver._ctx)
    roof_svd = {"kernel": "csvd_kernel", "bound": "alu", "achieved": svd_ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": svd_ach / fp32_peak, "traffic": dram_traffic("csvd_kernel", f"n{n}_r{r}"),
                "peak_source": f"FP32 FMA peak: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (one {nc_svd}-CTA "
                               f"cluster by design: its share is {nc_svd}/152 of this)",
                "cluster_ctas": nc_svd,
                "algorithmic_flops_per_launch": svd_flops, "avg_launch_us": svd_avg_us,
                "half_steps_per_launch": hsteps,
                "frac_of_its_sms": svd_ach / (fp32_peak * nc_svd / 152)}
    roof_pass["grid_blocks"] = pass_blocks
    roof_pass["tile_buffers"] = pass_bufs
    roofs = {"recon_vec_kernel": roof_recon, "pass_kernel": roof_pass, "csvd_kernel": roof_svd}
    # the kernel that takes the most of a step: the pass counts with the time it
    # adds after the SVD (its earlier part overlaps the SVD)
    share = {"csvd_kernel": per_step_us["csvd_kernel"], "pass_kernel": per_step_us["pass_kernel_after_svd"],
             "recon_vec_kernel": per_step_us["recon_vec_kernel"]}
    dominant = max(share, key=lambda kk: share[kk])

    e2e = None
    if a.e2e_steps > 0:
        Dh = torch.from_numpy(p.D).pin_memory()
        Lh = torch.empty((n, n), dtype=torch.float32).pin_memory()
        Sh = torch.empty((n, n), dtype=torch.float32).pin_memory()
        e2e_solver = ir.IRCUR(n, n, a.r, gamma=0.7, tol=1e-5, max_iter=100, resample=resample,
                              seed=a.seed + 1 + rank)
        ir.ircur_solve_host(e2e_solver._ctx, Dh, Lh, Sh)  # warm-up (allocates the device buffers)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        e_iters = 0
        for _ in range(a.e2e_steps):
            r2 = ir.ircur_solve_host(e2e_solver._ctx, Dh, Lh, Sh)
            e_iters += r2.iters
        el = time.perf_counter() - t0
        el, e_iters = aggregate(dist, world, el, e_iters, "cuda")
        e2e = {"value": e_iters / el, "unit": "iters/s", "h2d_bytes_per_step": 4 * n * n,
               "d2h_bytes_per_step": 8 * n * n, "ms_per_step": 1e3 * el / a.e2e_steps,
               "api": "ircur_solve_host (pinned host D in, dense L and S out)"}
        e2e_solver.close()
        # the same with Alg. 1's own output: the rank-r factors (L = A B; S = T_zeta(D - A B))
        f_solver = ir.IRCUR(n, n, a.r, gamma=0.7, tol=1e-5, max_iter=100, resample=resample, seed=a.seed + 1 + rank)
        Dd = torch.empty((n, n), dtype=torch.float32, device="cuda")
        Ah = torch.empty((n, a.r), dtype=torch.float32).pin_memory()
        Bh = torch.empty((a.r, n), dtype=torch.float32).pin_memory()

        # the step's copies alone, for comparison: D up, then L and S down (the
        # same pinned buffers and bytes, one copy each)
        def copies():
            c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            c0.record(stream)
            Dd.copy_(Dh, non_blocking=True)
            c1.record(stream)
            Lh.copy_(Dd, non_blocking=True)
            Sh.copy_(Dd, non_blocking=True)
            c2.record(stream)
            torch.cuda.synchronize()
            return c0.elapsed_time(c1), c1.elapsed_time(c2)

        copies()
        ct = [copies() for _ in range(3)]
        h2d_ms = float(np.median([u for u, _ in ct]))
        d2h_ms = float(np.median([v for _, v in ct]))
        e2e["copies_alone"] = {"h2d_ms": h2d_ms, "h2d_gb_per_s": 4 * n * n / (h2d_ms * 1e6),
                               "d2h_ms": d2h_ms, "d2h_gb_per_s": 8 * n * n / (d2h_ms * 1e6),
                               "ms": h2d_ms + d2h_ms,
                               "what": "pinned host buffers, D up then L and S down, CUDA events, no compute"}

        def host_factors():
            Dd.copy_(Dh, non_blocking=True)
            res_ = f_solver.solve(Dd)
            A_, B_ = f_solver.factors()
            Ah.copy_(A_, non_blocking=True)
            Bh.copy_(B_, non_blocking=True)
            torch.cuda.synchronize()
            return res_.iters

        host_factors()
        barrier()
        t0 = time.perf_counter()
        f_iters = sum(host_factors() for _ in range(a.e2e_steps))
        fel = time.perf_counter() - t0
        fel, f_iters = aggregate(dist, world, fel, f_iters, "cuda")
        e2e["factors_output"] = {"value": f_iters / fel, "unit": "iters/s", "h2d_bytes_per_step": 4 * n * n,
                                 "d2h_bytes_per_step": 8 * n * a.r, "ms_per_step": 1e3 * fel / a.e2e_steps,
                                 "api": "pinned host D in (torch copy), ircur_solve, ircur_get_factors, "
                                        "factors A (n x r) and B (r x n) out"}
        f_solver.close()

    # the other variant of Sec. 3.4 on the same D, for context (not the headline)
    other = "F" if resample else "R"
    osolver = ir.IRCUR(n, n, a.r, gamma=0.7, tol=1e-5, max_iter=100, resample=not resample, seed=a.seed + 1 + rank)
    for _ in range(2):
        osolver.solve(D)
    torch.cuda.synchronize()
    o0 = torch.cuda.Event(enable_timing=True)
    o1 = torch.cuda.Event(enable_timing=True)
    o0.record(stream)
    o_iters = 0
    for _ in range(3):
        o_iters += osolver.solve(D).iters
    o1.record(stream)
    torch.cuda.synchronize()
    other_line = {"variant": f"IRCUR-{other}", "time_to_tol_ms": o0.elapsed_time(o1) / 3,
                  "iters_per_solve": o_iters / 3}
    osolver.close()

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        c_iters, c_solves, c_el, _ = cpu_oracle_sample(p, a, a.cpu_seconds)
        cpu = {"value": c_iters / c_el, "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{c_solves} whole oracle solve(s) of the same workload (numpy FP64, "
                         f"{c_iters} iterations, {c_el:.1f} s), numpy/BLAS default threads",
               "time_to_tol_ms": 1e3 * c_el / c_solves}

    extras = {}
    if rank == 0 and world == 1 and not a.no_extras:
        from paper_2010_07422_gb300 import synth
        for key, fn in (("batched", bench_batched), ("adjoint", bench_adjoint), ("precision_variant", bench_precision),
                        ("streaming", bench_stream)):
            try:
                extras[key] = fn(ir, synth, stream)
            except Exception as exc:  # a secondary measurement must not cost the headline line
                extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
            torch.cuda.synchronize()

    if rank == 0:
        # per solve: setup, sampler, max|D| (+ D^T for IRCUR-R), zeta_0, the core's
        # D(I,J) (+ the two panel gathers for IRCUR-F); per iteration the core SVD and
        # the panel pass, launched for every iteration of each four-iteration graph
        # trip; the reconstruction
        launches_per_step = [5 + (2 if not resample else 0) + 2 * 4 * ((it + 3) // 4) + 1 for it in iters]
        line = {
            "metric": METRIC, "value": all_iters / (total_ms_max / 1e3), "unit": "iters/s",
            "n_gpus": world, "steps": a.steps, "warmup": max(3, a.warmup),
            "ms_per_step": total_ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(a), "n1": n, "n2": n, "r": a.r, "alpha": a.alpha,
                       "variant": a.variant, "nI": solver.nI, "nJ": solver.nJ,
                       "l2": "inputs larger than L2 (D is 400 MB; 1.2 GB streamed per step)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "time_to_tol_ms": float(np.mean(solve_ms)),
            "other_variant": other_line,
            "reconstruct_ms": float(np.mean(recon_ms)),
            "iters_per_solve": float(np.mean(iters)),
            "svd_steps_per_iter": svd_steps / max(1.0, my_iters),
            "flags": flags,
            "rel_err_vs_truth": rel_err_truth,
            "roofline": roofs[dominant],
            "roofline_other": {kk: vv for kk, vv in roofs.items() if kk != dominant},
            "kernel_us_per_step": per_step_us,
            "autotune": tune,
            "cur_to_svd_us": c2s_us,
            "timing_note": "kernel spans from the device clock (first block start to last block end) inside "
                           "the CUDA graph; the pass kernel is launched as a programmatic dependent of the "
                           "core SVD and overlaps it: pass_kernel is its whole launch span (used for its "
                           "roofline fraction), pass_kernel_after_svd the span from its first return of the "
                           "wait for the SVD; the reconstruction by CUDA events on the solver's stream",
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(sum(launches_per_step)),
            "clocks": clocks,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
