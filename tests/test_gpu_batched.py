"""GPU parity of the batched uneven-image solver against the oracle, image by image."""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, autotune, synth

pytestmark = pytest.mark.gpu
TOL = 2e-5
DEV = "cuda:0"


def _gpu(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _batch(sizes, lams, seed0, edge=()):
    fs, whs, wvs = [], [], []
    for m, (h, w) in enumerate(sizes):
        f = synth.shapes_image(h, w, seed=seed0 + m, n_shapes=max(1, h * w // 400))[1]
        fs.append(f)
        if m in edge:
            wh, wv = synth.edge_aware_weights(f, lams[m])
        else:
            wh = wv = None
        whs.append(wh)
        wvs.append(wv)
    return fs, whs, wvs


def _check(fs, whs, wvs, lams, y0s=None, max_iters=100, tol=1e-4):
    y0s = y0s or [None] * len(fs)
    xs, its, gaps, ok = _lib.tv2d_denoise_batched(
        [_gpu(f) for f in fs], lams, [_gpu(w) for w in whs], [_gpu(w) for w in wvs],
        [_gpu(y) for y in y0s], max_iters=max_iters, tol=tol)
    all_ok = True
    for m, f in enumerate(fs):
        xo, ito, tro, oko = oracle.tv2d_pd(f, lam=lams[m], w_h=whs[m], w_v=wvs[m], y0=y0s[m],
                                           max_iters=max_iters, tol=tol)
        assert its[m] == ito, (m, its[m], ito)
        assert np.abs(xs[m].cpu().numpy() - xo).max() <= TOL, m
        if ito:
            assert abs(gaps[m] - tro[-1]) <= 1e-6 + 1e-3 * abs(tro[-1])
        all_ok = all_ok and oko
    assert ok == all_ok
    return its


def test_mixed_sizes_weights_and_warm_starts():
    sizes = [(37, 50), (64, 64), (100, 33), (1, 40), (40, 1), (128, 96), (2, 2)]
    lams = [0.05, 0.1, 0.3, 0.2, 0.15, 0.25, 0.1]
    fs, whs, wvs = _batch(sizes, lams, seed0=10, edge=(1, 5))
    y0s = [None] * len(fs)
    y0s[2] = (0.02 * synth.shapes_image(100, 33, seed=99, n_shapes=5)[1]).astype(np.float32)
    its = _check(fs, whs, wvs, lams, y0s=y0s)
    assert len(set(its)) > 1  # images stop at their own iteration counts


def test_iteration_cap_and_fixed_iterations():
    sizes = [(48, 52), (30, 70)]
    lams = [0.2, 0.1]
    fs, whs, wvs = _batch(sizes, lams, seed0=40)
    _check(fs, whs, wvs, lams, max_iters=3, tol=0.0)
    _check(fs, whs, wvs, lams, max_iters=2, tol=1e-9)


def test_uneven_workload_sampled():
    """64 images, sizes uniform in 128x96 .. 2048x1536, lambda ~ U[0.05, 0.3],
    edge-aware weights: four images compared with the oracle."""
    sizes, lams = synth.uneven_image_sizes(64, seed=100)
    fs = [synth.shapes_image(h, w, seed=100 + m)[1] for m, (h, w) in enumerate(sizes)]
    ws = [synth.edge_aware_weights(f, lams[m]) for m, f in enumerate(fs)]
    xs, its, gaps, ok = _lib.tv2d_denoise_batched(
        [_gpu(f) for f in fs], lams, [_gpu(w[0]) for w in ws], [_gpu(w[1]) for w in ws],
        max_iters=200, tol=1e-4)
    assert ok and all(g <= 1e-4 for g in gaps)
    assert _lib.load().tv2d_batched_last_mode() in (0, 1)
    for m in (0, 17, 40, 63):
        xo, ito, tro, oko = oracle.tv2d_pd(fs[m], lam=lams[m], w_h=ws[m][0], w_v=ws[m][1],
                                           max_iters=200, tol=1e-4)
        assert its[m] == ito
        assert np.abs(xs[m].cpu().numpy() - xo).max() <= TOL


def test_autotune_runs_and_applies(tmp_path):
    params = autotune.autotune(path=str(tmp_path / "tune.json"))
    assert params["batched_warps"] in autotune.CHOICES_WPB
    assert params["coop_max_chains"] >= 1
    again = autotune.autotune(path=str(tmp_path / "tune.json"))  # from the cache
    assert again == params
    _lib.set_coop_max_chains(0)
    _lib.set_batched_warps(4)


def test_host_replay_matches_graph_loop():
    """The conditional-graph outer loop and its host replay give bitwise equal results."""
    sizes = [(64, 80), (33, 120), (96, 40)]
    lams = [0.1, 0.25, 0.05]
    fs, whs, wvs = _batch(sizes, lams, seed0=70, edge=(1,))
    runs = []
    try:
        for on in (1, 0):
            _lib.set_batched_graph(on)
            ys = [torch.empty(h, w, device=DEV) for h, w in sizes]
            xs, its, gaps, ok = _lib.tv2d_denoise_batched(
                [_gpu(f) for f in fs], lams, [_gpu(w) for w in whs], [_gpu(w) for w in wvs],
                max_iters=100, tol=1e-4, y_outs=ys)
            runs.append((xs, ys, its, gaps, _lib.load().tv2d_batched_last_mode()))
    finally:
        _lib.set_batched_graph(1)
    (xa, ya, ia, ga, ma), (xb, yb, ib, gb, mb) = runs
    assert mb == 0 and ma in (0, 1)
    assert ia == ib and ga == gb
    assert all(torch.equal(a, b) for a, b in zip(xa, xb))
    assert all(torch.equal(a, b) for a, b in zip(ya, yb))


@pytest.mark.parametrize("case", ["mixed", "cap"])
def test_thread_per_chain_path(case):
    """Batches above the warp-per-chain limit run one thread per chain (groups of 32 rows
    or columns of one image): forced here on small images, against the oracle."""
    try:
        _lib.set_coop_max_chains(1)
        if case == "mixed":
            sizes = [(37, 50), (64, 64), (100, 33), (1, 40), (40, 1), (128, 96), (2, 2), (70, 129)]
            lams = [0.05, 0.1, 0.3, 0.2, 0.15, 0.25, 0.1, 0.12]
            fs, whs, wvs = _batch(sizes, lams, seed0=110, edge=(1, 5, 7))
            y0s = [None] * len(fs)
            y0s[2] = (0.02 * synth.shapes_image(100, 33, seed=98, n_shapes=5)[1]).astype(np.float32)
            its = _check(fs, whs, wvs, lams, y0s=y0s)
            assert len(set(its)) > 1
        else:
            sizes = [(48, 52), (30, 70), (33, 31)]
            lams = [0.2, 0.1, 0.3]
            fs, whs, wvs = _batch(sizes, lams, seed0=140, edge=(0,))
            _check(fs, whs, wvs, lams, max_iters=3, tol=0.0)
    finally:
        _lib.set_coop_max_chains(0)
