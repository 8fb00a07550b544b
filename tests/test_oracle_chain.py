"""Pins of the FP64 chain oracle against facts fixed by eq. 1D-ROF (no GPU)."""
import os

import numpy as np
import pytest

import oracle
from paper_1502_07770_gb300 import synth
from tests import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chain_closed_forms.txt")


@pytest.mark.parametrize("case", range(len(pins.read_closed_forms(GOLDEN))))
def test_hand_derived_cases(case):
    c, w, x_ref, note = pins.read_closed_forms(GOLDEN)[case]
    x = oracle.chain_solve(c, w if len(w) else None, lam=0.0)
    np.testing.assert_allclose(x, x_ref, atol=1e-12, err_msg=note)


def test_brute_force_short_chains():
    rng = np.random.default_rng(0)
    for trial in range(150):
        n = int(rng.integers(1, 8))
        c = rng.normal(size=n) * rng.choice([0.1, 1.0, 10.0])
        w = rng.uniform(0.0, 1.5, size=n - 1)
        if trial % 5 == 0 and n > 1:
            w[rng.integers(0, n - 1)] = 0.0
        x = oracle.chain_solve(c, w)
        np.testing.assert_allclose(x, pins.brute_force_chain(c, w), atol=1e-10)


def test_bvls_dual_qp():
    rng = np.random.default_rng(1)
    for _ in range(60):
        n = int(rng.integers(2, 80))
        c = np.cumsum(rng.normal(size=n)) * 0.3
        w = rng.uniform(0.0, 2.0, size=n - 1)
        np.testing.assert_allclose(oracle.chain_solve(c, w), pins.bvls_chain(c, w), atol=1e-10)


@pytest.mark.parametrize("lam", [0.0, 0.05, 0.2, 3.0, 1e4])
def test_kkt_certificate_long(lam):
    y = synth.chain_batch(4, 25000, seed0=7).ravel().astype(np.float64)
    x = oracle.chain_solve(y, None, lam=lam)
    assert pins.kkt_residual(y, lam, x) < 1e-9


def test_kkt_random_weights_long():
    rng = np.random.default_rng(2)
    c = rng.normal(size=50000)
    w = rng.exponential(0.5, size=49999)
    x = oracle.chain_solve(c, w)
    assert pins.kkt_residual(c, w, x) < 1e-9


def test_closed_forms():
    rng = np.random.default_rng(3)
    c = rng.normal(size=300)
    np.testing.assert_allclose(oracle.chain_solve(c, None, lam=0.0), c, atol=1e-14)  # w = 0
    const = np.full(100, 0.37)
    np.testing.assert_allclose(oracle.chain_solve(const, None, lam=0.5), const, atol=1e-15)
    # w >= max_k |sum_{j<=k} (mean - c_j)| makes every edge fused: x = mean(c)
    bound = np.max(np.abs(np.cumsum(c.mean() - c)))
    np.testing.assert_allclose(oracle.chain_solve(c, None, lam=bound * 1.0001), c.mean(),
                               atol=1e-12)
    assert oracle.chain_solve(np.array([2.5]), None, lam=1.0)[0] == 2.5
    assert oracle.chain_solve(np.zeros(0), None, lam=1.0).shape == (0,)


def test_metamorphic():
    rng = np.random.default_rng(4)
    c = synth.piecewise_constant_chain(400, 9).astype(np.float64)
    w = rng.uniform(0.0, 0.4, size=399)
    x = oracle.chain_solve(c, w)
    # reversal of the chain
    np.testing.assert_allclose(oracle.chain_solve(c[::-1], w[::-1]), x[::-1], atol=1e-12)
    # translation and scaling
    np.testing.assert_allclose(oracle.chain_solve(c + 3.0, w), x + 3.0, atol=1e-12)
    np.testing.assert_allclose(oracle.chain_solve(2.5 * c, 2.5 * w), 2.5 * x, atol=1e-12)
    # mean preservation (u_n = 0)
    assert abs(x.sum() - c.sum()) < 1e-10
    # the prox is non-expansive
    c2 = c + rng.normal(scale=0.05, size=c.shape)
    x2 = oracle.chain_solve(c2, w)
    assert np.linalg.norm(x2 - x) <= np.linalg.norm(c2 - c) + 1e-12


def test_records_and_message_size():
    c = synth.piecewise_constant_chain(2000, 5).astype(np.float64)
    x, lo, hi, m = oracle.chain_solve(c, None, lam=0.2, return_records=True)
    assert np.all(lo <= hi + 1e-12)
    # the backward clip reproduces x from the records (Algorithm 2, backward pass)
    xb = np.empty_like(x)
    xb[-1] = x[-1]
    for i in range(len(x) - 2, -1, -1):
        xb[i] = min(max(xb[i + 1], lo[i]), hi[i])
    np.testing.assert_array_equal(xb, x)
    assert 2 <= m <= 2 * len(c) + 2
    # a steep ramp with a weight just below the all-fused threshold (about n^2/8)
    # keeps about one breakpoint per node: the message grows to about n/2
    n = 300
    _, _, _, m_big = oracle.chain_solve(-np.arange(float(n)), None, lam=n * n / 16.0,
                                        return_records=True)
    assert m_big >= n // 3


def test_batch_matches_single():
    y, off = synth.ragged_chain_batch([0, 1, 2, 17, 256, 5, 0, 1000], seed0=3)
    w = np.random.default_rng(5).uniform(0, 0.3, size=y.shape).astype(np.float32)
    xb = oracle.chain_solve_batch(y, off, w=w, nthreads=3)
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        xs = oracle.chain_solve(y[a:b], w[a:b - 1] if b - a > 1 else None)
        np.testing.assert_array_equal(xb[a:b], xs)


def _fd_grad(c, w, g, h=1e-6):
    out = np.empty_like(c)
    for j in range(len(c)):
        cp = c.copy(); cp[j] += h
        cm = c.copy(); cm[j] -= h
        out[j] = (g @ oracle.chain_solve(cp, w) - g @ oracle.chain_solve(cm, w)) / (2 * h)
    return out


def test_vjp_against_finite_differences():
    rng = np.random.default_rng(6)
    for trial in range(8):
        c = synth.piecewise_constant_chain(64, 100 + trial).astype(np.float64)
        w = np.full(63, 0.15)
        g = rng.normal(size=64)
        x = oracle.chain_solve(c, w)
        gc, gw = oracle.chain_vjp(x, g, with_w=True)
        np.testing.assert_allclose(gc, _fd_grad(c, w, g), atol=1e-6)
        h = 1e-6
        fdw = np.empty(63)
        for e in range(63):
            wp = w.copy(); wp[e] += h
            wm = w.copy(); wm[e] -= h
            fdw[e] = (g @ oracle.chain_solve(c, wp) - g @ oracle.chain_solve(c, wm)) / (2 * h)
        np.testing.assert_allclose(gw, fdw, atol=1e-6)


def test_jacobian_structure():
    c = synth.piecewise_constant_chain(50, 11).astype(np.float64)
    x = oracle.chain_solve(c, None, lam=0.2)
    J = np.stack([oracle.chain_vjp(x, e) for e in np.eye(50)], axis=0)
    np.testing.assert_allclose(J, J.T, atol=1e-15)            # symmetric
    np.testing.assert_allclose(J.sum(axis=1), 1.0, atol=1e-12)  # translation invariance
