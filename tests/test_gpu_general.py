"""GPU parity of the general convex chain solver (Sec. 4 with the quadratic unaries of
Sec. 4.1: curvature a_i, pairwise slopes w^-_i <= w^+_i) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 2e-5


def _gpu(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def _general_inputs(lengths, seed, unit_a=False):
    y, off = synth.ragged_chain_batch(lengths, seed0=seed)
    rng = np.random.default_rng(seed)
    n = y.size
    a = np.ones(n, np.float32) if unit_a else rng.uniform(0.5, 2.0, n).astype(np.float32)
    b = (a * y).astype(np.float32)  # targets in [0, 1]: x stays on the data's scale
    wlo = rng.uniform(-0.3, 0.05, n).astype(np.float32)
    whi = (wlo + rng.uniform(0.0, 0.4, n)).astype(np.float32)
    return a, b, wlo, whi, off


@pytest.mark.parametrize("split", [0, 1, 2])
def test_general_chains_against_oracle(split):
    lengths = [1, 2, 3, 31, 32, 63, 64, 65, 127, 300, 1000, 4097, 2, 64]
    a, b, wlo, whi, off = _general_inputs(lengths, seed=31)
    try:
        _lib.set_coop_split(split)
        x = _lib.chain_prox_general(_gpu(b), _gpu(wlo), _gpu(whi), a=_gpu(a),
                                    offsets=torch.from_numpy(off).to(DEV),
                                    max_len=max(lengths)).cpu().numpy()
    finally:
        _lib.set_coop_split(1)
    xr = oracle.chain_solve_general(a, b, wlo, whi, off)
    assert np.abs(x - xr).max() <= TOL


def test_unit_curvature_symmetric_matches_tv_l2():
    y = synth.chain_batch(256, 512, seed0=4)
    w = np.full(y.shape, 0.15, np.float32)
    x = _lib.chain_prox_general(_gpu(y), _gpu(-w), _gpu(w)).cpu().numpy()
    xt = _lib.chain_prox(_gpu(y), lam=0.15).cpu().numpy()
    assert np.abs(x - xt).max() <= 1e-6
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(257) * 512, lam=0.15).reshape(y.shape)
    assert np.abs(x - xr).max() <= TOL


def test_uniform_batch_and_linear_terms():
    rng = np.random.default_rng(7)
    B, n = 64, 200
    a = rng.uniform(0.5, 2.0, (B, n)).astype(np.float32)
    b = (a * rng.uniform(0, 1, (B, n))).astype(np.float32)
    beta = rng.normal(scale=0.2, size=(B, n)).astype(np.float32)
    x = _lib.chain_prox_general(_gpu(b), _gpu(beta), _gpu(beta), a=_gpu(a)).cpu().numpy()
    # w^- = w^+ = beta: x_i = (b_i + beta_i - beta_{i-1}) / a_i (beta_{-1} = beta_{n-1} = 0)
    bn = beta.astype(np.float64).copy()
    bn[:, -1] = 0.0
    bp = np.concatenate([np.zeros((B, 1)), beta[:, :-1].astype(np.float64)], axis=1)
    np.testing.assert_allclose(x, (b + bn - bp) / a, atol=TOL)


def test_general_overflow_path():
    # a steep ramp with wide symmetric bounds keeps ~n/2 breakpoints (more than 16/32 lanes)
    n = 400
    B = 8
    b = np.tile((-np.arange(n) / n).astype(np.float32), (B, 1))
    a = np.ones((B, n), np.float32)
    wlo = np.full((B, n), -n / 16.0, np.float32)
    whi = np.full((B, n), n / 16.0, np.float32)
    ws = _lib.workspace(_lib.load().tv_chain_workspace_size(B, n), DEV, "gen-overflow")
    x = _lib.chain_prox_general(_gpu(b), _gpu(wlo), _gpu(whi), a=_gpu(a), ws=ws).cpu().numpy()
    assert _lib.workspace_status(ws)[1] >= B
    xr = oracle.chain_solve_general(a.ravel(), b.ravel(), wlo.ravel(), whi.ravel(),
                                    np.arange(B + 1) * n).reshape(B, n)
    assert np.abs(x - xr).max() <= TOL


def test_general_halves_at_full_ring_capacity():
    """Half messages that peak at exactly 16 breakpoints (a 28-node steep ramp with heavy
    slopes, at either end) through the general chain halves, with a = 1 and
    [w-, w+] = [-w, w]: against the general oracle and against the TV-l2 oracle, which
    this case reduces to."""
    n = 80
    ys, wv = [], []
    for k in range(16):
        base = np.concatenate([(-np.arange(28) / 40.0),
                               np.random.default_rng(40 + k).uniform(0, 1, n - 28)])
        w = np.concatenate([np.full(28, 2.5), np.full(n - 28, 0.05)])
        if k % 2:
            base = base[::-1].copy()
            w = np.concatenate([w[:n - 1][::-1], [0.0]])
        ys.append(base)
        wv.append(w)
    b = np.concatenate(ys).astype(np.float32)
    w = np.concatenate(wv).astype(np.float32)
    a = np.ones_like(b)
    off = (np.arange(17) * n).astype(np.int64)
    x = _lib.chain_prox_general(_gpu(b), _gpu(-w), _gpu(w), a=_gpu(a),
                                offsets=torch.from_numpy(off).to(DEV), max_len=n).cpu().numpy()
    xg = oracle.chain_solve_general(a, b, -w, w, off)
    xt = oracle.chain_solve_batch(b, off, w=w)
    assert np.abs(x - xg).max() <= TOL
    assert np.abs(xg - xt).max() <= 1e-9
