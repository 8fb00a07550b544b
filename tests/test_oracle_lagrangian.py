"""Pins of the oracle's symmetric Lagrangian ROF solver (the (x_h, x_v, y) split of Sec. 6
with tau_k = tau0 / k) against the exact ROF minimiser (scipy BVLS on small images)."""
import numpy as np
import pytest

import oracle
from paper_1502_07770_gb300 import synth
from tests import pins


@pytest.mark.parametrize("edge_aware", [False, True])
def test_gap_bounds_and_convergence(edge_aware):
    f = synth.shapes_image(12, 10, 3, n_shapes=6)[1].astype(np.float64)
    lam = 0.1
    if edge_aware:
        w_h, w_v = synth.edge_aware_weights(f.astype(np.float32), lam)
        w_h, w_v = w_h.astype(np.float64), w_v.astype(np.float64)
    else:
        w_h, w_v = np.full((12, 9), lam), np.full((11, 10), lam)
    xs = pins.rof_exact(f, w_h, w_v)
    Ps = oracle.rof_primal(f, xs, w_h, w_v)
    N = f.size
    for k in (2, 8, 32, 128, 1024):
        x, it, tr, _ = oracle.tv2d_lagrangian(f, w_h=w_h, w_v=w_v, tau0=10.0, max_iters=k, tol=0.0,
                                              check_every=k)
        assert it == k
        G = tr[-1] * N
        P = oracle.rof_primal(f, x, w_h, w_v)
        # weak duality (D(y) <= P*) and 1-strong convexity: G >= P - P* >= |x - x*|^2 / 2
        assert G >= P - Ps - 1e-12
        assert P - Ps >= 0.5 * np.sum((x - xs) ** 2) - 1e-12
    assert np.abs(x - xs).max() < 1e-3


def test_stops_at_tolerance_and_agrees_with_the_accelerated_form():
    f = synth.shapes_image(64, 48, 1, n_shapes=20)[1]
    x, it, tr, ok = oracle.tv2d_lagrangian(f, lam=0.1, tau0=10.0, max_iters=400, tol=1e-4,
                                           check_every=5)
    assert ok and tr[-1] <= 1e-4 and it % 5 == 0
    checked = tr[~np.isnan(tr)]
    assert np.all(checked >= -1e-12) and np.all(checked[:-1] > 1e-4)
    # both forms solve the same strongly convex problem: per-pixel gaps 1e-4 bound the
    # distance to the minimiser by sqrt(2 G), so tighten both and compare
    xl, *_ = oracle.tv2d_lagrangian(f, lam=0.1, tau0=10.0, max_iters=3000, tol=1e-10,
                                    check_every=50)
    xp, *_ = oracle.tv2d_pd(f, lam=0.1, max_iters=400, tol=1e-12)
    assert np.abs(xl - xp).max() < 1e-3


def test_no_regulariser_returns_f():
    f = synth.shapes_image(10, 11, 4, n_shapes=6)[1].astype(np.float64)
    x, it, tr, ok = oracle.tv2d_lagrangian(f, lam=0.0, tau0=10.0, max_iters=3, tol=0.0,
                                           check_every=1)
    np.testing.assert_allclose(x, f, atol=1e-13)
    np.testing.assert_allclose(tr, 0.0, atol=1e-13)
