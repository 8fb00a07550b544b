"""GPU parity of the chain-prox backward (differentiable TV layer) against the oracle.

Workload of the differentiable-prox configuration: 4096 chains of 1024 nodes from
the step-signal generator, lambda = 0.15, loss = sum_i c_i x_i with c ~ N(0, 1).
The gradient is piecewise constant in y: it changes only where the segment
structure of the solution changes, which FP32 and FP64 may place differently at
(rare) near-degenerate jumps; such chains are counted and must stay rare, and the
gradient is compared on the others.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 2e-5


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _structure(x):
    return np.diff(x) == 0.0


@pytest.fixture(scope="module")
def cfg3():
    B, n = 4096, 1024
    y = synth.chain_batch(B, n, seed0=1000)
    c = synth.gaussian_vector(B * n, seed=7).reshape(B, n)
    return y, c


def test_config3_backward_against_oracle_vjp(cfg3):
    y, c = cfg3
    B, n = y.shape
    yg, cg = _gpu(y), _gpu(c)
    x = _lib.chain_prox(yg, lam=0.15)
    gy, _ = _lib.chain_prox_backward(x, cg)
    x_np, gy_np = x.cpu().numpy(), gy.cpu().numpy()
    # invariants on every chain: the Jacobian's columns sum to one, so sum(grad) = sum(c)
    np.testing.assert_allclose(gy_np.sum(axis=1, dtype=np.float64), c.sum(axis=1, dtype=np.float64),
                               atol=5e-3)
    sample = np.random.default_rng(0).choice(B, size=128, replace=False)
    xo = oracle.chain_solve_batch(y[sample].ravel(), np.arange(129) * n, lam=0.15).reshape(128, n)
    mismatched = 0
    for r, k in enumerate(sample):
        if not np.array_equal(_structure(xo[r]), _structure(x_np[k])):
            mismatched += 1
            continue
        go = oracle.chain_vjp(xo[r], c[k], fuse_tol=0.0)
        assert np.abs(go - gy_np[k]).max() <= TOL
    assert mismatched <= 2


def test_finite_differences_32_chains(cfg3):
    y, c = cfg3
    n = y.shape[1]
    h = 1e-6
    rows = np.arange(32)
    x = _lib.chain_prox(_gpu(y[rows]), lam=0.15)
    gy = _lib.chain_prox_backward(x, _gpu(c[rows]))[0].cpu().numpy()
    checked = 0
    for r in rows:
        y64 = y[r].astype(np.float64)
        base = oracle.chain_solve(y64, None, lam=0.15)
        pert = np.repeat(y64[None, :], 2 * n, axis=0)
        pert[np.arange(n), np.arange(n)] += h
        pert[n + np.arange(n), np.arange(n)] -= h
        xs = oracle.chain_solve_batch(pert.ravel(), np.arange(2 * n + 1) * n, lam=0.15).reshape(2 * n, n)
        fd = (xs[:n] @ c[r].astype(np.float64) - xs[n:] @ c[r].astype(np.float64)) / (2 * h)
        same = np.array([np.array_equal(_structure(xs[j]), _structure(base)) and
                         np.array_equal(_structure(xs[n + j]), _structure(base)) for j in range(n)])
        if not np.array_equal(_structure(base), _structure(x.cpu().numpy()[r])):
            continue
        np.testing.assert_allclose(gy[r][same], fd[same], atol=5e-5)
        checked += 1
    assert checked >= 30


def test_weight_gradients_against_oracle():
    rng = np.random.default_rng(3)
    B, n = 64, 300
    y = synth.chain_batch(B, n, seed0=50)
    w = rng.uniform(0.05, 0.3, size=y.shape).astype(np.float32)
    g = rng.normal(size=y.shape).astype(np.float32)
    x = _lib.chain_prox(_gpu(y), _gpu(w))
    gy, gw = _lib.chain_prox_backward(x, _gpu(g), with_w=True)
    x_np, gy_np, gw_np = x.cpu().numpy(), gy.cpu().numpy(), gw.cpu().numpy()
    xo = oracle.chain_solve_batch(y.ravel(), np.arange(B + 1) * n, w=w.ravel()).reshape(B, n)
    checked = 0
    for k in range(B):
        if not np.array_equal(_structure(xo[k]), _structure(x_np[k])):
            continue
        go, gwo = oracle.chain_vjp(xo[k], g[k], fuse_tol=0.0, with_w=True)
        assert np.abs(go - gy_np[k]).max() <= TOL
        assert np.abs(gwo - gw_np[k, :-1]).max() <= TOL
        checked += 1
    assert checked >= B - 2


def test_ragged_offsets_backward():
    lengths = [0, 1, 2, 31, 32, 33, 64, 65, 500, 1, 7]
    yv, off = synth.ragged_chain_batch(lengths, seed0=9)
    g = np.random.default_rng(1).normal(size=yv.shape).astype(np.float32)
    offd = _gpu(off)
    x = _lib.chain_prox(_gpu(yv), lam=0.2, offsets=offd, max_len=max(lengths))
    gy, _ = _lib.chain_prox_backward(x, _gpu(g), offsets=offd, max_len=max(lengths))
    x_np, gy_np = x.cpu().numpy(), gy.cpu().numpy()
    for k in range(len(lengths)):
        a, b = off[k], off[k + 1]
        if b > a:
            np.testing.assert_allclose(gy_np[a:b], oracle.chain_vjp(x_np[a:b].astype(np.float64), g[a:b],
                                                                    fuse_tol=0.0), atol=1e-6)


def test_long_chains_backward():
    """A batch with chains longer than the shared-memory records (4096 nodes): every
    chain's segment means then live in grad_y itself. Lengths around the 32-node step and
    the 128-node batch of steps; dL/dy and dL/dw against the oracle's VJP on the GPU's
    own segments."""
    lengths = [5000, 4097, 129, 128, 127, 33, 1, 0, 4100, 97]
    yv, off = synth.ragged_chain_batch(lengths, seed0=21)
    rng = np.random.default_rng(4)
    g = rng.normal(size=yv.shape).astype(np.float32)
    w = rng.uniform(0.05, 0.3, size=yv.shape).astype(np.float32)
    offd = _gpu(off)
    x = _lib.chain_prox(_gpu(yv), _gpu(w), offsets=offd, max_len=max(lengths))
    gy, gw = _lib.chain_prox_backward(x, _gpu(g), offsets=offd, max_len=max(lengths), with_w=True)
    x_np, gy_np, gw_np = x.cpu().numpy(), gy.cpu().numpy(), gw.cpu().numpy()
    for k in range(len(lengths)):
        a, b = off[k], off[k + 1]
        if b > a:
            go, gwo = oracle.chain_vjp(x_np[a:b].astype(np.float64), g[a:b], fuse_tol=0.0,
                                       with_w=True)
            np.testing.assert_allclose(gy_np[a:b], go, atol=1e-5)
            np.testing.assert_allclose(gw_np[a:b - 1], gwo, atol=1e-5)


def test_autograd_function():
    y = torch.from_numpy(synth.chain_batch(16, 200, seed0=3)).to(DEV).requires_grad_(True)
    w = torch.full((16, 200), 0.1, device=DEV, requires_grad=True)
    c = torch.randn(16, 200, device=DEV, generator=torch.Generator(DEV).manual_seed(0))
    x = _lib.chain_prox_diff(y, w)
    (x * c).sum().backward()
    gy, gw = _lib.chain_prox_backward(x.detach(), c, with_w=True)
    assert torch.equal(y.grad, gy) and torch.equal(w.grad, gw)
    # a Python-float weight: gradient to y only
    y2 = y.detach().clone().requires_grad_(True)
    (_lib.chain_prox_diff(y2, 0.1) * c).sum().backward()
    assert torch.allclose(y2.grad, gy, atol=1e-6)
