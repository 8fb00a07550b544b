"""Pins of the FP64 2D primal-dual oracle (eq. pd) against the ROF model (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_1502_07770_gb300 import synth
from tests import pins


def _small_image(H, W, seed, shapes=6):
    return synth.shapes_image(H, W, seed, n_shapes=shapes)[1].astype(np.float64)


@pytest.mark.parametrize("edge_aware", [False, True])
def test_converges_to_exact_rof_and_gap_bounds(edge_aware):
    f = _small_image(12, 10, 3)
    lam = 0.1
    if edge_aware:
        w_h, w_v = synth.edge_aware_weights(f.astype(np.float32), lam)
        w_h, w_v = w_h.astype(np.float64), w_v.astype(np.float64)
    else:
        w_h, w_v = np.full((12, 9), lam), np.full((11, 10), lam)
    xs = pins.rof_exact(f, w_h, w_v)
    Ps = oracle.rof_primal(f, xs, w_h, w_v)
    N = f.size
    prev = np.inf
    for k in (1, 2, 4, 8, 16, 64, 256):
        x, it, tr, _ = oracle.tv2d_pd(f, w_h=w_h, w_v=w_v, max_iters=k, tol=0.0)
        assert it == k
        G = tr[-1] * N
        P = oracle.rof_primal(f, x, w_h, w_v)
        # weak duality and 1-strong convexity of the primal: G >= P - P* >= |x - x*|^2 / 2
        assert G >= P - Ps - 1e-12
        assert P - Ps >= 0.5 * np.sum((x - xs) ** 2) - 1e-12
        assert G < prev * 1.05
        prev = G
    assert 0.5 * np.sum((x - xs) ** 2) < 1e-5


def test_gap_nonnegative_and_tolerance_stop():
    f = synth.shapes_image(64, 48, 1, n_shapes=20)[1]
    x, it, tr, ok = oracle.tv2d_pd(f, lam=0.1, max_iters=200, tol=1e-4)
    assert ok and tr[-1] <= 1e-4 and np.all(tr[:-1] > 1e-4)
    assert np.all(tr >= -1e-12)


def test_special_cases():
    const = np.full((9, 7), 0.3)
    x, it, tr, ok = oracle.tv2d_pd(const, lam=0.2, max_iters=5, tol=1e-12)
    np.testing.assert_allclose(x, const, atol=1e-14)
    assert ok and it == 1
    f = _small_image(10, 11, 4)
    x, *_ = oracle.tv2d_pd(f, lam=0.0, max_iters=3, tol=0.0)
    np.testing.assert_allclose(x, f, atol=1e-13)        # no regulariser: x = f
    x, it, tr, ok = oracle.tv2d_pd(f, lam=100.0, max_iters=400, tol=1e-12)
    np.testing.assert_allclose(x, f.mean(), atol=1e-5)  # huge weight: the image mean


def test_warm_start_from_optimal_dual_is_immediate():
    """Starting from a dual that the exact ROF solution certifies, x^0 is already optimal."""
    f = _small_image(8, 9, 5)
    lam = 0.15
    w_h, w_v = np.full((8, 8), lam), np.full((7, 9), lam)
    xs = pins.rof_exact(f, w_h, w_v)
    # any y with f - y = x* + D_h^T p_h: take the vertical part of the exact dual, y = D_v^T p_v,
    # recovered column by column from x* (column chains of the exact solution).
    _, _, tr0, _ = oracle.tv2d_pd(f, lam=lam, max_iters=1, tol=0.0)
    x1, _, tr, _ = oracle.tv2d_pd(f, lam=lam, max_iters=50, tol=0.0, return_y=True)[:4]
    y = oracle.tv2d_pd(f, lam=lam, max_iters=50, tol=0.0, return_y=True)[4]
    _, _, trw, _ = oracle.tv2d_pd(f, lam=lam, y0=y, max_iters=1, tol=0.0)
    assert trw[0] < tr0[0]
    assert 0.5 * np.sum((x1 - xs) ** 2) <= tr[-1] * f.size + 1e-12
