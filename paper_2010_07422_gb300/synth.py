"""Seeded synthetic workloads for IRCUR (D = L + S).

This module holds input generators only and none of the method's arithmetic;
the tests, the benchmark and the CPU oracle's callers all draw their inputs
from here, so the CUDA path and the oracle always see identical data.

Workloads (shapes and distributions of the paper's experiments, Sec. 4 and
the supplement's setup):

* ``planted``     -- L = W V^T with W, V i.i.d. N(0,1) of size n x r; S has
                     exactly round(alpha n1 n2) nonzeros on a uniformly drawn
                     support with values uniform in [-s E|L|, s E|L|], E|L|
                     taken as the empirical mean of |L|.  D = L + S rounded
                     to FP32.
* ``video_like``  -- a stand-in for the paper's surveillance videos (Table 1):
                     each column is a vectorised frame; rank-2 smooth
                     background times per-frame gains, moving rectangles as
                     the sparse foreground, small Gaussian noise, values in
                     [0, 1].
* ``random_subset`` -- a sorted uniform m-subset of [0, n) from numpy's PCG64,
                     for handing explicit index sets to both sides.
* ``planted_spectrum`` -- the ``planted`` recipe with L = Q1 diag(sigma) Q2^T
                     for orthonormal Q1, Q2 and a prescribed spectrum sigma
                     (ill-conditioned low-rank parts).
* ``lowrank_core_spectrum`` -- a low-rank D whose |I| x |J| core D(I,J), for
                     given index sets, has exactly the prescribed singular
                     values (narrow gaps and deficient ranks of the core).
* ``planted_device`` -- the ``planted`` recipe drawn directly in device memory
                     with torch's CUDA generator (FP32 throughout), for large
                     timing workloads whose values no oracle needs; the
                     batch recipe ``uneven_batch`` draws the shapes, ranks and
                     outlier fractions of a set of independent problems.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Planted:
    D: np.ndarray  # float32, n1 x n2, C-contiguous
    W: np.ndarray  # float64, n1 x r
    V: np.ndarray  # float64, n2 x r   (L = W V^T)
    s_pos: np.ndarray  # int64 flat positions of the outliers, sorted
    s_val: np.ndarray  # float64 outlier values
    mean_abs_L: float

    @property
    def shape(self):
        return self.D.shape

    def L_true(self):
        return self.W @ self.V.T

    def S_true(self):
        S = np.zeros(self.D.shape, np.float64)
        S.reshape(-1)[self.s_pos] = self.s_val
        return S

    def L_entries(self, rows, cols):
        return np.einsum("kt,kt->k", self.W[rows], self.V[cols])


def _distinct_positions(rng, total, k):
    """k distinct positions of [0, total), uniformly (an exchangeable draw:
    distinct values of an i.i.d. oversample, then a uniform k-subset)."""
    if k == 0:
        return np.zeros(0, np.int64)
    if k > total // 2:
        return np.sort(rng.permutation(total)[:k]).astype(np.int64)
    got = np.zeros(0, np.int64)
    while got.size < k:
        extra = rng.integers(0, total, size=int(1.25 * (k - got.size)) + 16, dtype=np.int64)
        got = np.sort(np.concatenate([got, extra]))
        got = got[np.concatenate([[True], got[1:] != got[:-1]])]  # sorted distinct values
    pick = rng.choice(got.size, size=k, replace=False)
    return np.sort(got[pick])


def planted(n1, n2, r, alpha, seed, outlier_scale=10.0, chunk_rows=2048):
    """Planted rank-r + alpha-sparse pair (supplement, setup for synthetic data)."""
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((n1, r))
    V = rng.standard_normal((n2, r))
    D = np.empty((n1, n2), np.float32)
    abs_sum = 0.0
    for i0 in range(0, n1, chunk_rows):
        blk = W[i0:i0 + chunk_rows] @ V.T
        abs_sum += float(np.abs(blk).sum())
        D[i0:i0 + chunk_rows] = blk  # rounded to FP32 below, after S is added
    mean_abs = abs_sum / (n1 * n2)
    k = int(round(alpha * n1 * n2))
    pos = _distinct_positions(rng, n1 * n2, k)
    half = outlier_scale * mean_abs
    val = rng.uniform(-half, half, size=k)
    rows, cols = np.divmod(pos, n2)
    # D = L + S in FP64 at the outlier positions, then FP32
    lv = np.einsum("kt,kt->k", W[rows], V[cols])
    D.reshape(-1)[pos] = (lv + val).astype(np.float32)
    # the non-outlier entries: FP64 L rounded once to FP32
    return Planted(D=D, W=W, V=V, s_pos=pos, s_val=val, mean_abs_L=mean_abs)


def _outliers_into(rng, D, W, V, alpha, outlier_scale, mean_abs):
    n1, n2 = D.shape
    k = int(round(alpha * n1 * n2))
    pos = _distinct_positions(rng, n1 * n2, k)
    half = outlier_scale * mean_abs
    val = rng.uniform(-half, half, size=k)
    rows, cols = np.divmod(pos, n2)
    lv = np.einsum("kt,kt->k", W[rows], V[cols])
    D.reshape(-1)[pos] = (lv + val).astype(np.float32)
    return pos, val


def planted_spectrum(n1, n2, sigmas, alpha, seed, outlier_scale=10.0):
    """Planted pair whose low-rank part has the singular values `sigmas`
    (times sqrt(n1 n2), so that entries are of order sigmas[0]):
    L = Q1 diag(s) Q2^T with Q1 (n1 x r), Q2 (n2 x r) orthonormal (QR of
    Gaussian matrices); outliers as in ``planted``."""
    rng = np.random.default_rng(seed)
    sig = np.asarray(sigmas, np.float64) * math.sqrt(n1 * n2)
    r = sig.size
    Q1, _ = np.linalg.qr(rng.standard_normal((n1, r)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n2, r)))
    W = Q1 * sig
    V = Q2
    L = W @ V.T
    mean_abs = float(np.abs(L).mean())
    D = L.astype(np.float32)
    pos, val = _outliers_into(rng, D, W, V, alpha, outlier_scale, mean_abs)
    return Planted(D=D, W=W, V=V, s_pos=pos, s_val=val, mean_abs_L=mean_abs)


def lowrank_core_spectrum(n1, n2, I, J, core_sigmas, seed):
    """D = W V^T (rank len(core_sigmas), FP32, no outliers) whose core D(I,J)
    is exactly Q1 diag(core_sigmas) Q2^T up to the FP32 rounding of D, for
    orthonormal Q1 (|I| x k), Q2 (|J| x k): the rows W(I,:) = Q1 diag(sigmas)
    and V(J,:) = Q2 are set, the other rows are Gaussian with the core's scale."""
    rng = np.random.default_rng(seed)
    s = np.asarray(core_sigmas, np.float64)
    k = s.size
    I = np.asarray(I, np.int64)
    J = np.asarray(J, np.int64)
    Q1, _ = np.linalg.qr(rng.standard_normal((I.size, k)))
    Q2, _ = np.linalg.qr(rng.standard_normal((J.size, k)))
    W = rng.standard_normal((n1, k)) * (s / math.sqrt(I.size))
    V = rng.standard_normal((n2, k)) / math.sqrt(J.size)
    W[I] = Q1 * s
    V[J] = Q2
    D = (W @ V.T).astype(np.float32)
    return Planted(D=D, W=W, V=V, s_pos=np.zeros(0, np.int64), s_val=np.zeros(0), mean_abs_L=float(np.abs(D).mean()))


def random_subset(n, m, seed):
    """Sorted uniform m-subset of [0, n) drawn with numpy's generator."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=m, replace=False)).astype(np.int64)


@dataclass
class Video:
    D: np.ndarray  # float32, (h*w) x frames, column = vectorised frame
    background: np.ndarray  # float64, rank-2 background (h*w) x frames
    fg_mask: np.ndarray  # bool, foreground support


def video_like(h, w, frames, seed, n_rects=(5, 20), noise_std=1e-3, fg_fraction=0.05):
    """Video-shaped D in [0, 1]: rank-2 background (two smooth images times
    slowly varying per-frame gains), 5-20 moving rectangles of random
    intensity covering about `fg_fraction` of the pixels, plus N(0, noise_std)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.linspace(0, 1, h), np.linspace(0, 1, w), indexing="ij")

    def smooth_image():
        img = np.zeros((h, w))
        for _ in range(4):
            fy, fx = rng.uniform(0.5, 3.0, 2)
            py, px = rng.uniform(0, 2 * math.pi, 2)
            img += rng.uniform(0.2, 1.0) * np.cos(2 * math.pi * fy * yy + py) * np.cos(2 * math.pi * fx * xx + px)
        img -= img.min()
        return img / max(img.max(), 1e-12)

    B1, B2 = smooth_image(), smooth_image()
    g1 = 0.55 + 0.02 * np.cumsum(rng.standard_normal(frames)) / math.sqrt(frames)
    g2 = 0.25 + 0.02 * np.cumsum(rng.standard_normal(frames)) / math.sqrt(frames)
    bg = np.outer(B1.reshape(-1), g1) + np.outer(B2.reshape(-1), g2)
    bg = np.clip(bg, 0.0, 0.85)
    D = bg.copy()
    mask = np.zeros_like(D, dtype=bool)
    k = int(rng.integers(n_rects[0], n_rects[1] + 1))
    area = fg_fraction * h * w / k
    for _ in range(k):
        rh = max(2, int(math.sqrt(area) * rng.uniform(0.6, 1.4)))
        rw = max(2, int(area / rh))
        y0, x0 = rng.uniform(0, h - rh), rng.uniform(0, w - rw)
        vy, vx = rng.uniform(-1.5, 1.5, 2) * (h / frames + 0.2)
        val = rng.uniform(0.0, 1.0)
        t = np.arange(frames)
        ys = ((y0 + vy * t) % max(1, h - rh)).astype(np.int64)
        xs = ((x0 + vx * t) % max(1, w - rw)).astype(np.int64)
        for f in range(frames):
            frame = D[:, f].reshape(h, w)
            fm = mask[:, f].reshape(h, w)
            frame[ys[f]:ys[f] + rh, xs[f]:xs[f] + rw] = val
            fm[ys[f]:ys[f] + rh, xs[f]:xs[f] + rw] = True
    D += noise_std * rng.standard_normal(D.shape)
    np.clip(D, 0.0, 1.0, out=D)
    return Video(D=D.astype(np.float32), background=bg, fg_mask=mask)


def planted_device(n1, n2, r, alpha, seed, outlier_scale=10.0, device="cuda", return_factors=False):
    """The ``planted`` recipe on the device: L = W V^T (W, V ~ N(0,1), FP32),
    round(alpha n1 n2) outliers on a uniform random support, values uniform in
    [-s mean|L|, s mean|L|].  Returns the n1 x n2 FP32 tensor D = L + S (and
    W, V when return_factors)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    W = torch.randn(n1, r, generator=g, device=device, dtype=torch.float32)
    V = torch.randn(n2, r, generator=g, device=device, dtype=torch.float32)
    D = W @ V.T
    half = outlier_scale * float(D.abs().mean())
    k = int(round(alpha * n1 * n2))
    pos = torch.randperm(n1 * n2, generator=g, device=device)[:k]
    val = (torch.rand(k, generator=g, device=device, dtype=torch.float32) * 2.0 - 1.0) * half
    D.view(-1).index_add_(0, pos, val)
    if return_factors:
        return D, W, V
    return D


def uneven_batch(count, seed, n_range=(500, 4000), r_range=(2, 10), alpha_range=(0.05, 0.3)):
    """Shapes of a batch of independent problems: n1, n2 uniform integers in
    n_range, r uniform in r_range (inclusive), alpha uniform in alpha_range."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n1, n2 = (int(x) for x in rng.integers(n_range[0], n_range[1] + 1, size=2))
        out.append(dict(n1=n1, n2=n2, r=int(rng.integers(r_range[0], r_range[1] + 1)),
                        alpha=float(rng.uniform(*alpha_range))))
    return out

