"""Small, fixed workloads for kernel profilers (one GPU, inputs resident).

    python profile_cases.py tv2d     [--reps R]   # 1024x1024 denoise, lambda 0.1
    python profile_cases.py chain    [--reps R] [--chains B] [--len N]
    python profile_cases.py backward [--reps R]   # 4096 x 1024 chain VJP
    python profile_cases.py net      [--reps R] [--grouped]  # warm-start inference 1024x1024
    python profile_cases.py train    [--reps R]   # one training step, 8 x 512x512
    python profile_cases.py batched  [--reps R]   # 16 uneven images, host-replayed loop
    python profile_cases.py l1       [--reps R]   # TV-l1 1024x1024, 10 iterations
    python profile_cases.py nonconvex [--reps R] [--chains B]  # B x 1482 x 126 cost volume

Each case runs its workload R times (after one untimed call) and prints one line. The
batched case forbids the conditional-graph loop so that every kernel is an ordinary
launch that a profiler can replay.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from paper_1502_07770_gb300 import _lib, learned, synth  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["tv2d", "chain", "backward", "net", "train", "batched", "l1", "nonconvex"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--chains", type=int, default=None,
                    help="chains (chain case, default 32768) or rows (nonconvex, default 1000)")
    ap.add_argument("--len", type=int, default=1024)
    ap.add_argument("--grouped", action="store_true",
                    help="net case: activations in the channel-group layout")
    a = ap.parse_args(argv)
    dev = torch.device("cuda:0")
    if a.case == "tv2d":
        f = torch.from_numpy(synth.shapes_image(1024, 1024, seed=0)[1]).to(dev)
        run = lambda: _lib.tv2d_denoise(f, lam=0.1, max_iters=200, tol=1e-4)
    elif a.case == "chain":
        base = synth.chain_batch(256, a.len, seed0=1000)
        y = torch.from_numpy(np.tile(base, (max(1, (a.chains or 32768) // 256), 1))).to(dev)
        x = torch.empty_like(y)
        run = lambda: _lib.chain_prox(y, lam=0.15, out=x)
    elif a.case == "backward":
        y = torch.from_numpy(synth.chain_batch(4096, 1024, seed0=1000)).to(dev)
        c = torch.from_numpy(synth.gaussian_vector(4096 * 1024, seed=7).reshape(4096, 1024)).to(dev)
        x = _lib.chain_prox(y, lam=0.15)
        run = lambda: _lib.chain_prox_backward(x, c)
    elif a.case in ("net", "train"):
        net = learned.load_weights(dev)
        if a.case == "net":
            f = torch.from_numpy(synth.shapes_image(1024, 1024, seed=0)[1]).to(dev)
            run = lambda: net.predict_dual(f, 0.1, grouped=a.grouped)
        else:
            fs, lams, ys = learned.make_dataset(range(10000, 10008), H=512, W=512, device=dev,
                                                tol=1e-4, max_iters=50)
            run = lambda: net.train_step(fs, lams, ys)
    elif a.case == "l1":
        f = torch.from_numpy(synth.salt_pepper_image(1024, 1024, seed=7)).to(dev)
        run = lambda: _lib.tv2d_denoise_l1(f, lam=0.55, tau=0.1, max_iters=10, tol=0.0,
                                           check_every=10)
    elif a.case == "nonconvex":
        rows = a.chains or 1000
        vol = torch.from_numpy(synth.stereo_cost_volume(rows, 1482, 126, seed=0)[0]).to(dev)
        run = lambda: _lib.chain_prox_nonconvex(vol, sl=-1.0, sr=1.0, w=0.1, C=0.8,
                                                max_breakpoints=512)
    else:
        _lib.set_batched_graph(False)
        sizes, lams = synth.uneven_image_sizes(16, seed=100)
        fs = [torch.from_numpy(synth.shapes_image(h, w, seed=100 + m)[1]).to(dev)
              for m, (h, w) in enumerate(sizes)]
        run = lambda: _lib.tv2d_denoise_batched(fs, lams, max_iters=200, tol=1e-4)
    run()
    torch.cuda.synchronize(dev)
    for _ in range(a.reps):
        run()
    torch.cuda.synchronize(dev)
    print(f"{a.case}: {a.reps} runs done")


if __name__ == "__main__":
    main()
