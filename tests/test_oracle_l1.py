"""Pins of the oracle's TV-l1 denoising (Sec. 6): the primal-dual iteration with row chains
of piecewise-quadratic unaries, against the exact LP optimum of TV(x) + ||x - f||_1."""
import numpy as np
import pytest

import oracle
from paper_1502_07770_gb300 import synth


def _lp_optimum(f, w_h, w_v):
    from scipy.optimize import linprog

    H, W = f.shape
    N = H * W
    idx = np.arange(N).reshape(H, W)
    edges = list(zip(idx[:, :-1].ravel(), idx[:, 1:].ravel(), np.asarray(w_h).ravel())) + \
        list(zip(idx[:-1].ravel(), idx[1:].ravel(), np.asarray(w_v).ravel()))
    m = len(edges)
    c = np.concatenate([np.zeros(N), np.ones(N), [e[2] for e in edges]])
    A, b = [], []
    fv = f.ravel()
    for i in range(N):  # t_i >= |x_i - f_i|
        r = np.zeros(2 * N + m); r[i], r[N + i] = 1, -1; A.append(r); b.append(fv[i])
        r = np.zeros(2 * N + m); r[i], r[N + i] = -1, -1; A.append(r); b.append(-fv[i])
    for q, (i, j, _) in enumerate(edges):  # s_q >= |x_j - x_i|
        r = np.zeros(2 * N + m); r[j], r[i], r[2 * N + q] = 1, -1, -1; A.append(r); b.append(0.0)
        r = np.zeros(2 * N + m); r[j], r[i], r[2 * N + q] = -1, 1, -1; A.append(r); b.append(0.0)
    res = linprog(c, A_ub=np.array(A), b_ub=np.array(b),
                  bounds=[(None, None)] * N + [(0, None)] * (N + m), method="highs")
    assert res.status == 0
    return res.fun


def _salt_pepper(H, W, seed, frac=0.15):
    rng = np.random.default_rng(seed)
    f = synth.shapes_image(H, W, seed, n_shapes=4)[1].astype(np.float64)
    m = rng.uniform(size=f.shape) < frac
    f[m] = rng.integers(0, 2, m.sum())
    return f


@pytest.mark.parametrize("edge_aware", [False, True])
def test_reaches_the_lp_optimum(edge_aware):
    f = _salt_pepper(8, 7, 1)
    lam = 0.3
    if edge_aware:
        w_h, w_v = synth.edge_aware_weights(f.astype(np.float32), lam)
        w_h, w_v = w_h.astype(np.float64), w_v.astype(np.float64)
    else:
        w_h, w_v = np.full((8, 6), lam), np.full((7, 7), lam)
    Ps = _lp_optimum(f, w_h, w_v)
    x, e = oracle.tv2d_l1(f, w_h=w_h, w_v=w_v, tau=0.3, iters=1500)
    assert np.all(e >= Ps - 1e-9)          # never below the optimum (x^k is feasible)
    assert e[-1] - Ps <= 1e-9


def test_special_cases():
    f = _salt_pepper(9, 8, 2)
    x, e = oracle.tv2d_l1(f, lam=0.0, tau=0.3, iters=3)
    np.testing.assert_allclose(x, f, atol=1e-14)   # no regulariser: x = f
    # a huge weight forces a constant image; the best constant is a median of f
    x, e = oracle.tv2d_l1(f, lam=50.0, tau=0.3, iters=3000)
    np.testing.assert_allclose(e[-1], np.abs(f - np.median(f)).sum(), atol=1e-6)
