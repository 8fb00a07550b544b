"""Pins of the oracle's non-convex chain DP (Sec. 3): continuous piecewise-linear unaries
and truncated TV min(w |d|, C), against exhaustive dynamic programming over a finite
candidate set that provably holds a minimiser, and against a linear program."""
import numpy as np
import pytest

import oracle


def _random_unary(rng, lo=0.0, hi=10.0, kmax=6):
    k = int(rng.integers(1, kmax + 1))
    lam = np.sort(rng.choice(np.arange(lo, hi + 0.25, 0.25), size=k, replace=False))
    val = rng.uniform(0.0, 3.0, k)
    return lam, val, -rng.uniform(0.5, 3.0), rng.uniform(0.5, 3.0)


def _eval(u, z):
    lam, val, sl, sr = u
    z = np.asarray(z, dtype=np.float64)
    v = np.interp(z, lam, val)
    v = np.where(z < lam[0], val[0] + sl * (z - lam[0]), v)
    return np.where(z > lam[-1], val[-1] + sr * (z - lam[-1]), v)


def _energy(us, w, C, x):
    e = sum(float(_eval(u, xi)) for u, xi in zip(us, x))
    d = np.abs(np.diff(x)) * np.asarray(w[:-1])
    return e + float(np.minimum(d, np.asarray(C[:-1])).sum())


def _discrete_dp(us, w, C, labels):
    """Exact minimum over x in labels^n (Viterbi)."""
    labels = np.asarray(labels, dtype=np.float64)
    cost = _eval(us[0], labels)
    for i in range(1, len(us)):
        pair = np.minimum(w[i - 1] * np.abs(labels[:, None] - labels[None, :]), C[i - 1])
        cost = (cost[:, None] + pair).min(axis=0) + _eval(us[i], labels)
    return float(cost.min())


@pytest.mark.parametrize("seed", range(8))
def test_plain_tv_equals_dp_over_the_unary_breakpoints(seed):
    # C = inf: the energy is linear on cells bounded by unary breakpoints and x_i = x_j, so
    # a minimiser takes every x_i at some unary's breakpoint
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    us = [_random_unary(rng) for _ in range(n)]
    w = rng.uniform(0.0, 2.0, n)
    C = np.full(n, np.inf)
    x, e = oracle.chain_solve_nonconvex(us, w, C)
    U = np.unique(np.concatenate([u[0] for u in us]))
    ref = _discrete_dp(us, w, C, U)
    assert abs(e[0] - ref) <= 1e-9 * max(1.0, abs(ref))
    assert abs(_energy(us, w, C, x) - e[0]) <= 1e-9 * max(1.0, abs(ref))


@pytest.mark.parametrize("seed", range(8))
def test_truncated_tv_equals_dp_over_shifted_breakpoints(seed):
    # uniform w, C: at a vertex every x_i is a unary breakpoint plus k C/w, |k| < n
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 6))
    us = [_random_unary(rng, kmax=4) for _ in range(n)]
    w = np.full(n, rng.uniform(0.3, 2.0))
    C = np.full(n, rng.uniform(0.2, 2.0))
    x, e = oracle.chain_solve_nonconvex(us, w, C)
    U = np.unique(np.concatenate([u[0] for u in us]))
    r = C[0] / w[0]
    cand = np.unique((U[:, None] + r * np.arange(-(n - 1), n)[None, :]).ravel())
    ref = _discrete_dp(us, w, C, cand)
    assert abs(e[0] - ref) <= 1e-9 * max(1.0, abs(ref))
    assert abs(_energy(us, w, C, x) - e[0]) <= 1e-9 * max(1.0, abs(ref))
    # and a finer grid never does better
    grid = np.linspace(-3.0, 13.0, 641)
    assert _discrete_dp(us, w, C, grid) >= e[0] - 1e-9


def test_convex_unaries_match_a_linear_program():
    from scipy.optimize import linprog

    rng = np.random.default_rng(7)
    n = 12
    us = []
    for _ in range(n):
        # a convex piecewise-linear unary: increasing slopes
        lam = np.sort(rng.uniform(0, 10, 4))
        slopes = np.sort(rng.uniform(-3, 3, 5))
        val = np.concatenate([[rng.uniform(0, 1)], np.zeros(3)])
        for k in range(3):
            val[k + 1] = val[k] + slopes[k + 1] * (lam[k + 1] - lam[k])
        us.append((lam, val, slopes[0], slopes[4]))
    w = rng.uniform(0.1, 1.5, n)
    x, e = oracle.chain_solve_nonconvex(us, w)
    # LP: t_i >= every affine piece of f_i, s_e >= |x_{e+1} - x_e|
    nv = 2 * n + (n - 1)
    c = np.concatenate([np.zeros(n), np.ones(n), w[:-1]])
    A, b = [], []
    for i, (lam, val, sl, sr) in enumerate(us):
        slopes = [sl] + [(val[k + 1] - val[k]) / (lam[k + 1] - lam[k]) for k in range(3)] + [sr]
        anchors = [0] + list(range(4))
        for s, k in zip(slopes, anchors):
            row = np.zeros(nv); row[i] = s; row[n + i] = -1
            A.append(row); b.append(s * lam[k] - val[k])
    for q in range(n - 1):
        for sg in (1, -1):
            row = np.zeros(nv); row[q + 1] = sg; row[q] = -sg; row[2 * n + q] = -1
            A.append(row); b.append(0.0)
    res = linprog(c, A_ub=np.array(A), b_ub=np.array(b), bounds=[(None, None)] * nv,
                  method="highs")
    assert res.status == 0
    assert abs(e[0] - res.fun) <= 1e-8 * max(1.0, abs(res.fun))


def test_special_cases():
    rng = np.random.default_rng(3)
    n = 9
    us = [_random_unary(rng) for _ in range(n)]
    # w = 0 or C = 0: the nodes decouple
    sep = sum(float(u[1].min()) for u in us)
    for w, C in ((np.zeros(n), np.full(n, np.inf)), (np.ones(n), np.zeros(n))):
        x, e = oracle.chain_solve_nonconvex(us, w, C)
        assert abs(e[0] - sep) <= 1e-12
    # a huge C is plain TV
    w = rng.uniform(0.1, 1.0, n)
    _, e_inf = oracle.chain_solve_nonconvex(us, w)
    _, e_big = oracle.chain_solve_nonconvex(us, w, np.full(n, 1e3))
    assert abs(e_inf[0] - e_big[0]) <= 1e-9
    # reversing the chain, or mirroring every unary (z -> -z), keeps the optimum
    _, e_rev = oracle.chain_solve_nonconvex(us[::-1], np.concatenate([w[:-1][::-1], [0.0]]))
    mir = [(-u[0][::-1], u[1][::-1], -u[3], -u[2]) for u in us]
    _, e_mir = oracle.chain_solve_nonconvex(mir, w)
    assert abs(e_rev[0] - e_inf[0]) <= 1e-9 and abs(e_mir[0] - e_inf[0]) <= 1e-9
    # a single node: its minimum
    x, e = oracle.chain_solve_nonconvex(us[:1], w[:1])
    assert abs(e[0] - us[0][1].min()) <= 1e-12 and x[0] == us[0][0][np.argmin(us[0][1])]


def test_batch_offsets():
    rng = np.random.default_rng(5)
    lens = [3, 1, 0, 6]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    us = [_random_unary(rng) for _ in range(off[-1])]
    w = rng.uniform(0, 1, off[-1])
    C = rng.uniform(0.2, 1.0, off[-1])
    x, e = oracle.chain_solve_nonconvex(us, w, C, off)
    for k in range(len(lens)):
        s, t = off[k], off[k + 1]
        xs, es = oracle.chain_solve_nonconvex(us[s:t], w[s:t], C[s:t]) if t > s else (x[s:t], [0.0])
        np.testing.assert_array_equal(x[s:t], xs)
        assert e[k] == es[0]


@pytest.mark.parametrize("C", [np.inf, 3.0])
def test_grid_unaries_equal_dp_over_the_label_grid(C):
    # cost-volume unaries: breakpoints at the integer labels 0..L-1, steep ends; with C/w
    # an integer every vertex lies on the (extended) integer grid
    rng = np.random.default_rng(11)
    n, L = 40, 24
    lab = np.arange(L, dtype=np.float64)
    us = []
    for i in range(n):
        d0 = rng.uniform(0, L - 1)
        val = np.minimum(np.abs(lab - d0) / 4.0, 1.0) + 0.3 * rng.uniform(size=L)
        us.append((lab, val, -5.0, 5.0))
    w = np.full(n, 0.5)
    Cs = np.full(n, C)
    x, e = oracle.chain_solve_nonconvex(us, w, Cs)
    ext = np.arange(-(n - 1) * 6, L + (n - 1) * 6, dtype=np.float64)
    ref = _discrete_dp(us, w, Cs, ext)
    assert abs(e[0] - ref) <= 1e-9 * abs(ref)
    assert abs(_energy(us, w, Cs, x) - e[0]) <= 1e-9 * abs(ref)
