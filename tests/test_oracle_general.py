"""Pins of the oracle's general convex chain (Sec. 4 and Sec. 4.1: unaries a_i x^2/2 - b_i x,
pairwise w^-_i d / w^+_i d on d = x_{i+1} - x_i), none of which reuses its arithmetic
except the reduction to the TV-l2 chain."""
import itertools

import numpy as np

import oracle


def _random_chain(rng, n, lo=-0.4, hi=0.4):
    a = rng.uniform(0.5, 2.0, n)
    b = rng.normal(0.0, 1.0, n)
    w1 = rng.uniform(lo, hi, n)
    w2 = rng.uniform(lo, hi, n)
    return a, b, np.minimum(w1, w2), np.maximum(w1, w2)


def _kkt_residual(a, b, wlo, whi, x):
    """Optimality of x: u_i = sum_{k<=i} (a_k x_k - b_k) is the dual on edge i; need
    u_{n-1} = 0 and u_i in the subdifferential of f_i at x_{i+1} - x_i."""
    u = np.cumsum(a * x - b)
    res = abs(u[-1])
    d = np.diff(x)
    for i in range(len(x) - 1):
        if d[i] > 1e-12:
            res = max(res, abs(u[i] - whi[i]))
        elif d[i] < -1e-12:
            res = max(res, abs(u[i] - wlo[i]))
        else:
            res = max(res, wlo[i] - u[i], u[i] - whi[i], 0.0)
    return res


def _brute_force(a, b, wlo, whi):
    """Enumerate fused / up / down per edge; segment values from the duals at its ends."""
    n = len(b)
    found = []
    for pat in itertools.product((0, 1, -1), repeat=n - 1):
        x = np.empty(n)
        start, u_left, ok = 0, 0.0, True
        for i in range(n):
            if i == n - 1 or pat[i] != 0:
                u_right = 0.0 if i == n - 1 else (whi[i] if pat[i] == 1 else wlo[i])
                seg = slice(start, i + 1)
                x[seg] = (b[seg].sum() + u_right - u_left) / a[seg].sum()
                u = u_left  # interior duals of the fused segment
                for k in range(start, i):
                    u += a[k] * x[k] - b[k]
                    if u < wlo[k] - 1e-12 or u > whi[k] + 1e-12:
                        ok = False
                start, u_left = i + 1, u_right
        if not ok:
            continue
        if all((pat[i] == 1 and x[i + 1] > x[i]) or (pat[i] == -1 and x[i + 1] < x[i])
               for i in range(n - 1) if pat[i] != 0):
            found.append(x)
    return found


def test_reduces_to_the_tv_l2_chain():
    rng = np.random.default_rng(0)
    c = rng.uniform(0, 1, 300)
    w = rng.uniform(0, 0.3, 300)
    x = oracle.chain_solve_general(np.ones(300), c, -w, w)
    np.testing.assert_allclose(x, oracle.chain_solve(c, w[:-1]), atol=1e-12)


def test_kkt_certificate_on_long_random_chains():
    rng = np.random.default_rng(1)
    for n, (lo, hi) in ((2000, (-0.4, 0.4)), (1500, (-0.1, 0.6)), (800, (-2.0, 2.0))):
        a, b, wlo, whi = _random_chain(rng, n, lo, hi)
        x = oracle.chain_solve_general(a, b, wlo, whi)
        assert _kkt_residual(a, b, wlo, whi, x) < 1e-9


def test_brute_force_small_chains():
    rng = np.random.default_rng(2)
    for n in range(1, 8):
        for _ in range(6):
            a, b, wlo, whi = _random_chain(rng, n, -0.8, 0.8)
            x = oracle.chain_solve_general(a, b, wlo, whi)
            sols = _brute_force(a, b, wlo, whi)
            assert len(sols) >= 1
            np.testing.assert_allclose(x, sols[0], atol=1e-10)


def test_linear_pairwise_terms_have_a_closed_form():
    # w^- = w^+ = beta: sum beta_i (x_{i+1} - x_i) = sum_i x_i (beta_{i-1} - beta_i)
    rng = np.random.default_rng(3)
    n = 50
    a = rng.uniform(0.5, 2.0, n)
    b = rng.normal(size=n)
    beta = rng.normal(scale=0.3, size=n)
    x = oracle.chain_solve_general(a, b, beta, beta)
    bb = np.concatenate([[0.0], beta[:-1]])
    bn = beta.copy()
    bn[-1] = 0.0
    np.testing.assert_allclose(x, (b + bn - bb) / a, atol=1e-12)


def test_uniform_curvature_is_a_rescaled_tv_l2_chain():
    rng = np.random.default_rng(4)
    c = rng.uniform(0, 1, 200)
    w = rng.uniform(0, 0.3, 200)
    alpha = 2.5
    x = oracle.chain_solve_general(np.full(200, alpha), alpha * c, -alpha * w, alpha * w)
    np.testing.assert_allclose(x, oracle.chain_solve(c, w[:-1]), atol=1e-12)


def test_large_weights_fuse_everything():
    rng = np.random.default_rng(5)
    a, b, _, _ = _random_chain(rng, 40)
    x = oracle.chain_solve_general(a, b, np.full(40, -1e3), np.full(40, 1e3))
    np.testing.assert_allclose(x, np.full(40, b.sum() / a.sum()), atol=1e-12)


def test_batch_offsets():
    rng = np.random.default_rng(6)
    lens = [0, 1, 5, 30, 2]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    a, b, wlo, whi = _random_chain(rng, off[-1])
    x = oracle.chain_solve_general(a, b, wlo, whi, off)
    for k in range(len(lens)):
        s, e = off[k], off[k + 1]
        if e > s:
            np.testing.assert_allclose(x[s:e], oracle.chain_solve_general(a[s:e], b[s:e], wlo[s:e],
                                                                          whi[s:e]), atol=0)
