"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module draws random numbers and builds arrays; it contains none of the
total-variation arithmetic (no message passing, no proximal steps, no gap).
Every generator draws in float64 from numpy's PCG64 and returns float32 arrays,
so both sides of a parity test consume bit-identical inputs.

Workload shapes follow the experiments of Sec. 6 of the paper (noisy piecewise-
constant 1D signals as in the step-function experiment of Sec. 6.1, and noisy
piecewise-constant 2D images as in the ROF experiment of Sec. 6.1); the paper's
own test image and signal lengths are not available, so these stand in for them.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def piecewise_constant_chain(n: int, seed: int, seg_lo: int = 8, seg_hi: int = 64,
                             noise: float = 0.1) -> np.ndarray:
    """One noisy step signal of length ``n``.

    Segment lengths are drawn uniformly from the integers ``seg_lo..seg_hi``,
    segment levels uniformly from [0, 1], and i.i.d. Gaussian noise of standard
    deviation ``noise`` is added (the step-function workload of Sec. 6.1).
    """
    rng = _rng(seed)
    out = np.empty(n, dtype=np.float64)
    pos = 0
    while pos < n:
        length = int(rng.integers(seg_lo, seg_hi + 1))
        out[pos:pos + length] = rng.uniform(0.0, 1.0)
        pos += length
    out += rng.normal(0.0, noise, size=n)
    return out.astype(np.float32)


def chain_batch(num_chains: int, n: int, seed0: int = 0, **kw) -> np.ndarray:
    """``num_chains`` independent step signals of length ``n``, chain ``k`` seeded
    with ``seed0 + k``; returned as a C-contiguous (num_chains, n) float32 array."""
    out = np.empty((num_chains, n), dtype=np.float32)
    for k in range(num_chains):
        out[k] = piecewise_constant_chain(n, seed0 + k, **kw)
    return out


def ragged_chain_batch(lengths, seed0: int = 0, **kw):
    """Chains of the given lengths concatenated into one float32 vector, plus the
    int64 CSR offsets (length ``len(lengths) + 1``)."""
    lengths = [int(v) for v in lengths]
    offsets = np.zeros(len(lengths) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    y = np.empty(int(offsets[-1]), dtype=np.float32)
    for k, n in enumerate(lengths):
        if n:
            y[offsets[k]:offsets[k + 1]] = piecewise_constant_chain(n, seed0 + k, **kw)
    return y, offsets


def shapes_image(H: int, W: int, seed: int, n_shapes: int = 200, noise: float = 0.1,
                 background: float = 0.5) -> tuple[np.ndarray, np.ndarray]:
    """A noisy image of random axis-aligned rectangles and disks.

    Background ``background``; ``n_shapes`` shapes painted in order, each a
    rectangle (sides uniform in [W/32, W/4] and [H/32, H/4]) or a disk (radius
    uniform in [W/64, W/8]) with a uniform centre and a level uniform in [0, 1].
    Returns ``(clean, noisy)`` as float32 (H, W) arrays; the noisy one adds
    i.i.d. Gaussian noise of standard deviation ``noise`` and is not clipped.
    """
    rng = _rng(seed)
    img = np.full((H, W), background, dtype=np.float64)
    rr = np.arange(H, dtype=np.float64)[:, None]
    cc = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(n_shapes):
        level = rng.uniform(0.0, 1.0)
        cy = rng.uniform(0.0, H)
        cx = rng.uniform(0.0, W)
        if rng.uniform() < 0.5:
            hh = 0.5 * rng.uniform(H / 32.0, H / 4.0)
            hw = 0.5 * rng.uniform(W / 32.0, W / 4.0)
            y0, y1 = int(max(0, np.floor(cy - hh))), int(min(H, np.ceil(cy + hh)))
            x0, x1 = int(max(0, np.floor(cx - hw))), int(min(W, np.ceil(cx + hw)))
            img[y0:y1, x0:x1] = level
        else:
            rad = rng.uniform(W / 64.0, W / 8.0)
            y0, y1 = int(max(0, np.floor(cy - rad))), int(min(H, np.ceil(cy + rad + 1)))
            x0, x1 = int(max(0, np.floor(cx - rad))), int(min(W, np.ceil(cx + rad + 1)))
            sub = (rr[y0:y1] - cy) ** 2 + (cc[:, x0:x1] - cx) ** 2 <= rad * rad
            img[y0:y1, x0:x1][sub] = level
    noisy = img + rng.normal(0.0, noise, size=(H, W))
    return img.astype(np.float32), noisy.astype(np.float32)


def salt_pepper_image(H: int, W: int, seed: int, frac: float = 0.25) -> np.ndarray:
    """The noisy shapes image (``n_shapes`` = max(4, H W / 400)) with a fraction ``frac``
    of its pixels replaced by 0 or 1 (impulse noise; 25 % is the degradation of the
    TV-l1 experiment of Sec. 6).
    float32 (H, W)."""
    f = shapes_image(H, W, seed, n_shapes=max(4, H * W // 400))[1]
    rng = _rng(seed)
    m = rng.uniform(size=f.shape) < frac
    f[m] = rng.integers(0, 2, int(m.sum()))
    return f.astype(np.float32)


def stereo_cost_volume(H: int, W: int, L: int, seed: int, slope: float = 0.25,
                       trunc: float = 1.0, noise: float = 0.3,
                       outliers: float = 0.1) -> tuple[np.ndarray, np.ndarray]:
    """A synthetic matching-cost volume standing in for a stereo data term (Sec. 6):
    a disparity map of random slanted planes on rectangles and ellipses (levels in
    [0, L-1]), and per pixel the non-convex cost c(d) = min(slope |d - d*|, trunc) +
    U[0, noise] at the integer disparities d = 0..L-1, plus, at a fraction ``outliers`` of
    the pixels, a false minimum of depth 0.5 at a uniform disparity. Returns
    ``(cost (H, W, L) float32, d* (H, W) float32)``."""
    rng = _rng(seed)
    d = np.full((H, W), 0.5 * (L - 1))
    rr = np.arange(H, dtype=np.float64)[:, None]
    cc = np.arange(W, dtype=np.float64)[None, :]
    for _ in range(max(4, H * W // 4000)):
        level = rng.uniform(0.0, L - 1.0)
        gy, gx = rng.uniform(-0.05, 0.05, 2)
        cy, cx = rng.uniform(0.0, H), rng.uniform(0.0, W)
        hh, hw = 0.5 * rng.uniform(H / 16.0, H / 3.0), 0.5 * rng.uniform(W / 16.0, W / 3.0)
        rect = rng.uniform() < 0.5
        y0, y1 = int(max(0, np.floor(cy - hh))), int(min(H, np.ceil(cy + hh) + 1))
        x0, x1 = int(max(0, np.floor(cx - hw))), int(min(W, np.ceil(cx + hw) + 1))
        if y1 <= y0 or x1 <= x0:
            continue
        ry, rx = rr[y0:y1] - cy, cc[:, x0:x1] - cx
        if rect:
            m = (np.abs(ry) <= hh) & (np.abs(rx) <= hw)
        else:
            m = ry ** 2 / hh ** 2 + rx ** 2 / hw ** 2 <= 1.0
        sub = d[y0:y1, x0:x1]
        sub[m] = (level + gy * ry + gx * rx)[m]
    d = np.clip(d, 0.0, L - 1.0)
    cost = np.empty((H, W, L), dtype=np.float32)
    out = rng.uniform(size=(H, W)) < outliers
    fd = rng.integers(0, L, size=(H, W))
    lab = np.arange(L, dtype=np.float32)[None, :]
    d32 = d.astype(np.float32)
    for r in range(H):  # row by row, in FP32, to bound the temporaries
        c = np.minimum(np.float32(slope) * np.abs(lab - d32[r, :, None]), np.float32(trunc))
        c += np.float32(noise) * rng.random((W, L), dtype=np.float32)
        o = np.flatnonzero(out[r])
        if o.size:
            c[o] -= np.maximum(0.0, 0.5 - slope * np.abs(lab - fd[r, o, None])).astype(np.float32)
        cost[r] = c
    return cost, d.astype(np.float32)


def edge_aware_weights(f: np.ndarray, lam: float, scale: float = 0.2):
    """Per-edge weights ``lam * exp(-|f_i - f_j| / scale)`` of a float32 image.

    Returns ``(w_h, w_v)``: ``w_h`` of shape (H, W-1) for the edge between
    pixels (r, c) and (r, c+1), ``w_v`` of shape (H-1, W) for the edge between
    (r, c) and (r+1, c); both float32, computed in float64 from ``f``.
    """
    f64 = f.astype(np.float64)
    w_h = lam * np.exp(-np.abs(np.diff(f64, axis=1)) / scale)
    w_v = lam * np.exp(-np.abs(np.diff(f64, axis=0)) / scale)
    return w_h.astype(np.float32), w_v.astype(np.float32)


def uneven_image_sizes(count: int, seed: int, w_range=(128, 2048), h_range=(96, 1536)):
    """``count`` image sizes (H, W) with W and H drawn independently and uniformly
    from the given integer ranges, plus per-image lambda uniform in [0.05, 0.3]."""
    rng = _rng(seed)
    Ws = rng.integers(w_range[0], w_range[1] + 1, size=count)
    Hs = rng.integers(h_range[0], h_range[1] + 1, size=count)
    lams = rng.uniform(0.05, 0.3, size=count)
    return [(int(h), int(w)) for h, w in zip(Hs, Ws)], [float(v) for v in lams]


def gaussian_vector(n: int, seed: int) -> np.ndarray:
    """i.i.d. N(0, 1) float32 vector (the loss weights of the differentiable-prox workload)."""
    return _rng(seed).normal(0.0, 1.0, size=n).astype(np.float32)


def warm_start_sample(H: int, W: int, seed: int, lam_range=(0.05, 0.3)):
    """One sample of the learned warm-start workload: the noisy ``shapes_image`` of
    ``seed`` and a lambda uniform in ``lam_range`` drawn from an independent stream
    (PCG64 seeded with ``seed + 2**40``). Returns ``(noisy float32 (H, W), lambda)``."""
    _, noisy = shapes_image(H, W, seed)
    lam = float(_rng(seed + (1 << 40)).uniform(lam_range[0], lam_range[1]))
    return noisy, lam
