"""GPU parity of the 2D primal-dual ROF solver (eq. pd with row/column chain proxes)
against the FP64 oracle running the same iteration."""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
TOL = 2e-5
DEV = "cuda:0"


def _gpu(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _both(f, lam=0.1, w_h=None, w_v=None, y0=None, max_iters=50, tol=1e-4):
    xg, it, gap, ok = _lib.tv2d_denoise(_gpu(f), lam=lam, w_h=_gpu(w_h), w_v=_gpu(w_v),
                                        y0=_gpu(y0), max_iters=max_iters, tol=tol)
    xo, ito, tro, oko = oracle.tv2d_pd(f, lam=lam, w_h=w_h, w_v=w_v, y0=y0,
                                       max_iters=max_iters, tol=tol)
    return xg.cpu().numpy(), it, gap, ok, xo, ito, tro, oko


@pytest.mark.parametrize("shape", [(96, 80), (77, 45), (33, 129), (1, 50), (50, 1), (1, 1)])
def test_converged_parity(shape):
    H, W = shape
    f = synth.shapes_image(H, W, seed=3, n_shapes=max(1, H * W // 300))[1]
    xg, it, gap, ok, xo, ito, tro, oko = _both(f)
    assert ok == oko and it == ito
    assert np.abs(xg - xo).max() <= TOL
    if it > 0:
        assert abs(gap - tro[-1]) <= 1e-6 + 1e-3 * abs(tro[-1])


@pytest.mark.parametrize("iters", [0, 1, 2, 3, 8])
def test_fixed_iteration_parity(iters):
    """Same iterates for a fixed count (tol = 0), odd and even: exercises the buffer swap."""
    f = synth.shapes_image(64, 96, seed=5, n_shapes=20)[1]
    xg, it, gap, ok, xo, ito, tro, oko = _both(f, max_iters=iters, tol=0.0)
    assert it == ito == iters and not ok and not oko
    assert np.abs(xg - xo).max() <= TOL
    if iters:
        assert abs(gap - tro[-1]) <= 1e-6 + 1e-3 * abs(tro[-1])


def test_edge_aware_weights_and_warm_start():
    f = synth.shapes_image(100, 70, seed=7, n_shapes=30)[1]
    w_h, w_v = synth.edge_aware_weights(f, 0.2)
    y0 = (0.05 * synth.shapes_image(100, 70, seed=8, n_shapes=10)[1]).astype(np.float32)
    for a, b in ((w_h, w_v), (w_h, None), (None, w_v)):
        xg, it, gap, ok, xo, ito, tro, oko = _both(f, lam=0.15, w_h=a, w_v=b, y0=y0)
        assert ok == oko and it == ito
        assert np.abs(xg - xo).max() <= TOL


def test_special_images():
    const = np.full((40, 40), 0.3, np.float32)
    xg, it, gap, ok = _lib.tv2d_denoise(_gpu(const), lam=0.2, max_iters=10, tol=1e-6)
    assert ok and it == 1
    np.testing.assert_allclose(xg.cpu().numpy(), const, atol=1e-6)
    f = synth.shapes_image(30, 20, seed=2, n_shapes=5)[1]
    xg, *_ = _lib.tv2d_denoise(_gpu(f), lam=0.0, max_iters=3, tol=0.0)
    np.testing.assert_allclose(xg.cpu().numpy(), f, atol=1e-6)


def test_config1_full_size():
    """1024x1024, 200 shapes, lambda 0.1, to per-pixel gap 1e-4: the benchmark workload."""
    f = synth.shapes_image(1024, 1024, seed=0)[1]
    xg, it, gap, ok, xo, ito, tro, oko = _both(f, lam=0.1, max_iters=200, tol=1e-4)
    assert ok and oko and it == ito
    assert gap <= 1e-4
    assert np.abs(xg - xo).max() <= TOL


def test_chain_split_modes_agree():
    """The 2D solve with middle-rooted chains (two halves of a warp: default; two warps)
    and with one warp per chain from one end: same iteration count, results within FP32
    rounding of each other."""
    _, f = synth.shapes_image(200, 150, seed=5, n_shapes=40)
    ft = torch.from_numpy(f).to("cuda:0")
    out = []
    try:
        for split in (1, 2, 0):
            _lib.set_coop_split(split)
            out.append(_lib.tv2d_denoise(ft, lam=0.15, max_iters=100, tol=1e-4))
    finally:
        _lib.set_coop_split(1)
    for x, it, gap, ok in out:
        assert ok and it == out[0][1]
        assert (x - out[0][0]).abs().max().item() <= 2e-5


def test_programmatic_launch_gives_identical_results():
    """The 2D solver's kernels launched with a programmatic dependency on their
    predecessor (each waits in hardware for the previous grid before reading) give
    bitwise the same iterate, iteration count and gap as plain stream order."""
    _, f = synth.shapes_image(256, 320, seed=5, n_shapes=60)
    ft = torch.from_numpy(f).to(DEV)
    wh = torch.from_numpy(np.full((256, 319), 0.08, np.float32)).to(DEV)
    out = {}
    try:
        for on in (True, False):
            _lib.set_programmatic_launch(on)
            for name, kw in (("uniform", {}), ("weights", {"w_h": wh})):
                x, it, gap, ok = _lib.tv2d_denoise(ft, lam=0.1, max_iters=40, tol=1e-4, **kw)
                assert ok
                out[(on, name)] = (x.cpu().numpy(), it, gap)
    finally:
        _lib.set_programmatic_launch(True)
    for name in ("uniform", "weights"):
        a, b = out[(True, name)], out[(False, name)]
        assert a[1] == b[1] and a[2] == b[2]
        assert np.array_equal(a[0], b[0])
