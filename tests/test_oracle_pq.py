"""Pins of the oracle's chain with piecewise-quadratic unaries (Sec. 4.2):
a_i x^2/2 - b_i x + alpha_i |x - f_i| with TV weights w_i."""
import numpy as np
import pytest

import oracle


def _random(rng, n, alpha_hi=0.5, w_hi=0.4):
    a = rng.uniform(0.5, 2.0, n)
    b = a * rng.uniform(0, 1, n)
    alpha = rng.uniform(0, alpha_hi, n)
    f = rng.uniform(0, 1, n)
    w = rng.uniform(0, w_hi, n)
    return a, b, alpha, f, w


def _certificate(a, b, alpha, f, w, x, tol=1e-9):
    """Optimality of x by an LP feasibility problem over the free subgradients: v_i in
    [-1, 1] at nodes with x_i = f_i (else sign(x_i - f_i)); the edge duals
    u_i = sum_{k<=i} (a_k x_k - b_k + alpha_k v_k) must vanish at the end and lie in
    w_i * subdifferential of |x_{i+1} - x_i|."""
    from scipy.optimize import linprog

    n = len(x)
    kink = np.abs(x - f) <= 1e-12
    vfix = np.where(kink, 0.0, np.sign(x - f))
    free = np.flatnonzero(kink)
    m = len(free)
    base = np.cumsum(a * x - b + alpha * vfix)          # u without the free terms
    M = np.zeros((n, m))                                  # d u_i / d v_free
    for j, i in enumerate(free):
        M[i:, j] = alpha[i]
    A_ub, b_ub, A_eq, b_eq = [], [], [M[n - 1]], [-base[n - 1]]
    d = np.diff(x)
    for i in range(n - 1):
        if d[i] > 1e-12:
            A_eq.append(M[i]); b_eq.append(w[i] - base[i])
        elif d[i] < -1e-12:
            A_eq.append(M[i]); b_eq.append(-w[i] - base[i])
        else:
            A_ub.append(M[i]); b_ub.append(w[i] - base[i] + tol)
            A_ub.append(-M[i]); b_ub.append(w[i] + base[i] + tol)
    if m == 0:
        ok_eq = all(abs(be) <= 1e-8 for be in b_eq)
        ok_ub = all(bu >= -1e-8 for bu in b_ub)
        return ok_eq and ok_ub
    # equalities with a small slack, as two inequalities
    for row, rhs in zip(A_eq, b_eq):
        A_ub.append(row); b_ub.append(rhs + tol)
        A_ub.append(-row); b_ub.append(-rhs + tol)
    res = linprog(np.zeros(m), A_ub=np.array(A_ub), b_ub=np.array(b_ub), bounds=[(-1, 1)] * m,
                  method="highs")
    return res.status == 0


def test_no_l1_term_is_the_quadratic_chain():
    rng = np.random.default_rng(0)
    a, b, _, f, w = _random(rng, 300)
    x = oracle.chain_solve_pq(a, b, np.zeros(300), f, w)
    np.testing.assert_allclose(x, oracle.chain_solve_general(a, b, -w, w), atol=1e-12)


def test_no_tv_is_a_soft_threshold():
    rng = np.random.default_rng(1)
    a, b, alpha, f, _ = _random(rng, 200)
    x = oracle.chain_solve_pq(a, b, alpha, f, np.zeros(200))
    lo, hi = (b - alpha) / a, (b + alpha) / a
    np.testing.assert_allclose(x, np.where(hi < f, hi, np.where(lo > f, lo, f)), atol=1e-14)


@pytest.mark.parametrize("n", [2, 5, 40, 300])
def test_optimality_certificate(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        a, b, alpha, f, w = _random(rng, n)
        x = oracle.chain_solve_pq(a, b, alpha, f, w)
        assert _certificate(a, b, alpha, f, w, x)
        # and a wrong answer fails it
        y = x.copy()
        y[n // 2] += 1e-3
        assert not _certificate(a, b, alpha, f, w, y)


def test_large_l1_weight_returns_f():
    rng = np.random.default_rng(3)
    a, b, _, f, w = _random(rng, 50)
    alpha = np.abs(a * f - b) + 2 * w.max() + 0.1
    np.testing.assert_allclose(oracle.chain_solve_pq(a, b, alpha, f, w), f, atol=0)


def test_batch_offsets():
    rng = np.random.default_rng(4)
    lens = [1, 7, 0, 33, 2]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    a, b, alpha, f, w = _random(rng, off[-1])
    x = oracle.chain_solve_pq(a, b, alpha, f, w, off)
    for k in range(len(lens)):
        s, e = off[k], off[k + 1]
        if e > s:
            np.testing.assert_array_equal(x[s:e], oracle.chain_solve_pq(a[s:e], b[s:e], alpha[s:e],
                                                                        f[s:e], w[s:e]))
