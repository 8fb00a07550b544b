"""GPU parity of the non-convex chain DP (Sec. 3: piecewise-linear unaries, truncated TV)
against the oracle. A minimiser need not be unique, so the optimum energy is compared,
and the GPU's x is checked to reach it (its energy evaluated in FP64)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _rel_ok(a, b, rel=1e-5, abs_=1e-4):
    return abs(a - b) <= abs_ + rel * abs(b)


def _random_unary(rng, lo=0.0, hi=10.0, kmax=6):
    k = int(rng.integers(1, kmax + 1))
    lam = np.sort(rng.choice(np.arange(lo, hi + 0.25, 0.25), size=k, replace=False))
    val = rng.uniform(0.0, 3.0, k)
    return lam, val, -rng.uniform(0.5, 3.0), rng.uniform(0.5, 3.0)


def _eval(u, z):
    lam, val, sl, sr = u
    if len(lam) == 0:
        return 0.0
    if z < lam[0]:
        return val[0] + sl * (z - lam[0])
    if z > lam[-1]:
        return val[-1] + sr * (z - lam[-1])
    return float(np.interp(z, lam, val))


def _energy(us, w, C, x):
    e = sum(_eval(u, float(xi)) for u, xi in zip(us, x))
    d = np.abs(np.diff(np.asarray(x, dtype=np.float64))) * np.asarray(w[:-1], dtype=np.float64)
    return e + float(np.minimum(d, np.asarray(C[:-1], dtype=np.float64)).sum())


def _csr(us):
    lens = [len(u[0]) for u in us]
    uoff = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ulam = np.concatenate([np.asarray(u[0], np.float32) for u in us] + [np.zeros(1, np.float32)])
    uval = np.concatenate([np.asarray(u[1], np.float32) for u in us] + [np.zeros(1, np.float32)])
    sl = np.array([u[2] for u in us], np.float32)
    sr = np.array([u[3] for u in us], np.float32)
    return uoff, ulam, uval, sl, sr


def _f32(us):
    """The unaries as the GPU sees them (FP32 values widened to FP64)."""
    return [(np.asarray(u[0], np.float32).astype(np.float64),
             np.asarray(u[1], np.float32).astype(np.float64),
             float(np.float32(u[2])), float(np.float32(u[3]))) for u in us]


def _t(a, dtype=None):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).to(DEV)


def _check_batch(us, w, C, off, x, e):
    us = _f32(us)
    w = np.asarray(w, np.float32).astype(np.float64)
    C = np.asarray(C, np.float32).astype(np.float64)
    off = np.asarray(off, dtype=np.int64)
    xo, eo = oracle.chain_solve_nonconvex(us, w, C, off)
    for k in range(len(off) - 1):
        s, t = off[k], off[k + 1]
        assert _rel_ok(e[k], eo[k]), (k, e[k], eo[k])
        if t > s:
            ex = _energy(us[s:t], w[s:t], C[s:t], x[s:t])
            assert ex >= eo[k] - 1e-9 * max(1.0, abs(eo[k]))
            assert _rel_ok(ex, eo[k]), (k, ex, eo[k])


def _status():
    st, _ = _lib.workspace_status(_lib.workspace(1, DEV, "nonconvex"))
    return st


@pytest.mark.parametrize("truncated", [False, True])
def test_random_unaries_ragged_batch(truncated):
    rng = np.random.default_rng(1 if truncated else 0)
    lens = [1, 2, 0, 7, 40, 33, 64, 100, 3, 129, 0, 250]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    N = int(off[-1])
    us = [_random_unary(rng) for _ in range(N)]
    w = rng.uniform(0.0, 2.0, N).astype(np.float32)
    C = (rng.uniform(0.1, 3.0, N) if truncated else np.full(N, np.inf)).astype(np.float32)
    uoff, ulam, uval, sl, sr = _csr(us)
    x, e = _lib.chain_prox_nonconvex(_t(uval), uoff=_t(uoff), ulam=_t(ulam), sl=_t(sl), sr=_t(sr),
                                     w=_t(w), C=_t(C), offsets=_t(off), max_len=max(lens),
                                     max_breakpoints=256)
    assert _status() == _lib.TV_OK
    _check_batch(us, w, C, off, x.cpu().numpy(), e.cpu().numpy())


@pytest.mark.parametrize("C", [float("inf"), 0.6])
def test_cost_volume_chains(C):
    L = 64
    cost, _ = synth.stereo_cost_volume(24, 300, L, seed=2)
    wv = np.float32(0.2)
    x, e = _lib.chain_prox_nonconvex(_t(cost), sl=-1.0, sr=1.0, w=float(wv), C=C,
                                     max_breakpoints=512)
    assert _status() == _lib.TV_OK
    lab = np.arange(L, dtype=np.float64)
    us = [(lab, cost[r, i].astype(np.float64), -1.0, 1.0) for r in range(24) for i in range(300)]
    N = 24 * 300
    _check_batch(us, np.full(N, wv), np.full(N, C), np.arange(25) * 300, x.cpu().numpy(),
                 e.cpu().numpy())


def test_edge_weights_and_per_node_truncation_on_a_cost_volume():
    L = 40
    cost, _ = synth.stereo_cost_volume(8, 257, L, seed=3)
    rng = np.random.default_rng(4)
    N = 8 * 257
    w = rng.uniform(0.0, 0.5, N).astype(np.float32)
    C = rng.uniform(0.0, 2.0, N).astype(np.float32)
    C[::17] = 0.0
    x, e = _lib.chain_prox_nonconvex(_t(cost), sl=-2.0, sr=0.5, w=_t(w), C=_t(C),
                                     max_breakpoints=256)
    assert _status() == _lib.TV_OK
    lab = np.arange(L, dtype=np.float64)
    us = [(lab, cost[r, i].astype(np.float64), -2.0, 0.5) for r in range(8) for i in range(257)]
    _check_batch(us, w, C, np.arange(9) * 257, x.cpu().numpy(), e.cpu().numpy())


def test_decoupled_and_single_node_chains():
    rng = np.random.default_rng(5)
    us = [_random_unary(rng) for _ in range(50)]
    uoff, ulam, uval, sl, sr = _csr(us)
    ref = sum(float(u[1].min()) for u in _f32(us))
    for w, C in ((0.0, float("inf")), (1.0, 0.0)):  # the nodes decouple
        x, e = _lib.chain_prox_nonconvex(_t(uval), uoff=_t(uoff), ulam=_t(ulam), sl=_t(sl),
                                         sr=_t(sr), w=w, C=C, max_breakpoints=64)
        assert _rel_ok(float(e[0]), ref, abs_=1e-5)
    # fifty chains of one node: each its own argmin
    off = np.arange(51, dtype=np.int64)
    x, e = _lib.chain_prox_nonconvex(_t(uval), uoff=_t(uoff), ulam=_t(ulam), sl=_t(sl), sr=_t(sr),
                                     w=0.5, offsets=_t(off), max_len=1, max_breakpoints=64)
    xs, es = x.cpu().numpy(), e.cpu().numpy()
    for k, u in enumerate(_f32(us)):
        assert es[k] == pytest.approx(u[1].min(), abs=1e-6)
        assert xs[k] == np.float32(u[0][np.argmin(u[1])])


def test_capacity_overflow_is_reported():
    rng = np.random.default_rng(6)
    # the first chain's messages hold at most its 60 unary breakpoints; the second
    # chain's first unary alone has 200
    small = [_random_unary(rng, kmax=2) for _ in range(30)]
    big = [(np.arange(200, dtype=np.float64), rng.uniform(0, 1, 200), -1.0, 1.0) for _ in range(30)]
    off = np.array([0, 30, 60], dtype=np.int64)
    uoff, ulam, uval, sl, sr = _csr(small + big)
    x, e = _lib.chain_prox_nonconvex(_t(uval), uoff=_t(uoff), ulam=_t(ulam), sl=_t(sl), sr=_t(sr),
                                     w=0.3, offsets=_t(off), max_len=30, max_breakpoints=128)
    assert _status() == _lib.TV_ERR_CAPACITY
    xs, es = x.cpu().numpy(), e.cpu().numpy()
    assert np.isnan(es[1]) and np.all(np.isnan(xs[30:]))
    _check_batch(small, np.full(30, 0.3), np.full(30, np.inf), [0, 30], xs[:30], es[:1])


def test_invalid_arguments():
    vol = _t(np.zeros((2, 5, 4), np.float32))
    for kw in ({"sl": 0.5}, {"sr": -0.5}, {"w": -1.0}, {"C": -1.0}, {"max_breakpoints": 0},
               {"max_breakpoints": 3}):
        args = dict(sl=-1.0, sr=1.0, w=0.1, C=float("inf"), max_breakpoints=64)
        args.update(kw)
        with pytest.raises(_lib.TVError):
            _lib.chain_prox_nonconvex(vol, **args)


def test_full_size_rows_sampled():
    # a cost volume of the size of the paper's stereo pair (1000 rows of 1482 pixels, 126
    # disparities) solved in one launch; 12 rows checked against the oracle
    H, W, L = 1000, 1482, 126
    cost, _ = synth.stereo_cost_volume(H, W, L, seed=0)
    x, e = _lib.chain_prox_nonconvex(_t(cost), sl=-1.0, sr=1.0, w=0.1, C=0.8,
                                     max_breakpoints=512)
    assert _status() == _lib.TV_OK
    xs, es = x.cpu().numpy().reshape(H, W), e.cpu().numpy()
    lab = np.arange(L, dtype=np.float64)
    for r in np.random.default_rng(7).choice(H, 12, replace=False):
        us = [(lab, cost[r, i].astype(np.float64), -1.0, 1.0) for i in range(W)]
        _check_batch(us, np.full(W, 0.1), np.full(W, 0.8), [0, W], xs[r], es[r:r + 1])
