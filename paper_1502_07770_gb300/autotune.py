"""Autotuner for the launch choices of the TV library.

Two choices are measured on the running GPU and applied through the C ABI:
  * the largest batch of chains solved with one warp per chain (latency-bound
    batches) rather than one thread per chain (throughput-bound batches): the
    crossover is timed on uniform batches of 256- and 1024-node chains;
  * the warps per block of the persistent kernels of the batched 2D solver.
Results are cached as JSON keyed by the GPU name and library version, in
``$TV_AUTOTUNE_CACHE`` or ``~/.cache/tv_gb300/autotune.json``.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import _lib, synth

CHOICES_WPB = (2, 4, 8)
BATCHES = (512, 1024, 2048, 4096, 8192)
LENGTHS = (256, 1024)
FORCE_COOP = 1 << 40
FORCE_THREAD = 1


def cache_path() -> str:
    return os.environ.get("TV_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tv_gb300",
                                       "autotune.json"))


def cache_key(device=0) -> str:
    import torch
    return f"{torch.cuda.get_device_name(device)}|tv{_lib.load().tv_version()}"


def _time_ms(fn, reps=5, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def choose_crossover(timings):
    """Largest batch at which the warp kernel is at least as fast as the thread
    kernel for every measured length; timings: {(B, n): (warp_ms, thread_ms)}."""
    best = 0
    for B in sorted({b for b, _ in timings}):
        rows = [timings[(b, n)] for (b, n) in timings if b == B]
        if all(w <= t for w, t in rows):
            best = B
        else:
            break
    return best


def measure(device=0):
    import torch
    dev = torch.device("cuda", device)
    timings = {}
    for n in LENGTHS:
        base = synth.chain_batch(256, n, seed0=1000)
        for B in BATCHES:
            y = torch.from_numpy(np.tile(base, (B // 256, 1))).to(dev)
            x = torch.empty_like(y)
            res = []
            for force in (FORCE_COOP, FORCE_THREAD):
                _lib.set_coop_max_chains(force)
                res.append(_time_ms(lambda: _lib.chain_prox(y, lam=0.15, out=x)))
            timings[(B, n)] = tuple(res)
    _lib.set_coop_max_chains(0)
    crossover = choose_crossover(timings)
    # warps per block of the batched solver, on a small uneven batch
    sizes, lams = synth.uneven_image_sizes(6, seed=5, w_range=(128, 768), h_range=(96, 576))
    imgs = [torch.from_numpy(synth.shapes_image(h, w, seed=200 + i, n_shapes=40)[1]).to(dev)
            for i, (h, w) in enumerate(sizes)]
    wpb_ms = {}
    for wpb in CHOICES_WPB:
        _lib.set_batched_warps(wpb)
        wpb_ms[wpb] = _time_ms(lambda: _lib.tv2d_denoise_batched(imgs, lams, max_iters=100,
                                                                 tol=1e-4), reps=3, warm=1)
    best_wpb = min(wpb_ms, key=wpb_ms.get)
    return {"coop_max_chains": int(max(crossover, 1)), "batched_warps": int(best_wpb),
            "chain_timings_ms": {f"{b}x{n}": list(v) for (b, n), v in timings.items()},
            "batched_warps_ms": {str(k): v for k, v in wpb_ms.items()}}


def apply(params):
    _lib.set_coop_max_chains(int(params["coop_max_chains"]))
    _lib.set_batched_warps(int(params["batched_warps"]))


def load_cache(path=None):
    path = path or cache_path()
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def save_cache(data, path=None):
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(device=0, force=False, path=None):
    """Tuned parameters for this GPU (measured once, then read from the cache), applied."""
    key = cache_key(device)
    data = load_cache(path)
    if force or key not in data:
        data[key] = measure(device)
        save_cache(data, path)
    apply(data[key])
    return data[key]
