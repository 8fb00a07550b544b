"""GPU parity of the chain solver with piecewise-quadratic unaries (Sec. 4.2) against the
FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 2e-5


def _gpu(v):
    return None if v is None else torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).to(DEV)


def _inputs(lengths, seed, repeated=False):
    rng = np.random.default_rng(seed)
    n = int(sum(lengths))
    off = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    a = rng.uniform(0.5, 2.0, n).astype(np.float32)
    b = (a * rng.uniform(0, 1, n)).astype(np.float32)
    al = rng.uniform(0, 0.5, n).astype(np.float32)
    f = rng.uniform(0, 1, n).astype(np.float32)
    if repeated:
        f = (np.round(f * 8) / 8).astype(np.float32)
    w = rng.uniform(0, 0.4, n).astype(np.float32)
    return a, b, al, f, w, off


@pytest.mark.parametrize("repeated", [False, True])
def test_ragged_chains_against_oracle(repeated):
    lengths = [1, 2, 3, 31, 32, 33, 64, 300, 1000, 2, 17]
    a, b, al, f, w, off = _inputs(lengths, 3, repeated)
    x = _lib.chain_prox_pq(_gpu(b), _gpu(f), a=_gpu(a), alpha=_gpu(al), w=_gpu(w),
                           offsets=torch.from_numpy(off).to(DEV), max_len=max(lengths)).cpu().numpy()
    xr = oracle.chain_solve_pq(a, b, al, f, w, off)
    assert np.abs(x - xr).max() <= TOL


def test_tv_l1_row_prox_shape():
    """The row proximal map of TV-l1: alpha = 1, a = 1/tau, b = xi/tau on noisy image rows."""
    _, img = synth.shapes_image(64, 512, seed=2, n_shapes=40)
    tau = 0.5
    xi = img + np.random.default_rng(1).normal(0, 0.05, img.shape).astype(np.float32)
    b = (xi / tau).astype(np.float32)
    x = _lib.chain_prox_pq(_gpu(b), _gpu(img), a=_gpu(np.full(img.shape, 1 / tau)), alpha=1.0,
                           lam=0.3).cpu().numpy()
    n = img.shape[1]
    xr = oracle.chain_solve_pq(np.full(img.size, 1 / tau), b.ravel(), np.ones(img.size), img.ravel(),
                               np.full(img.size, 0.3), np.arange(img.shape[0] + 1) * n)
    assert np.abs(x.ravel() - xr).max() <= TOL


def test_reductions():
    rng = np.random.default_rng(9)
    y = synth.chain_batch(64, 256, seed0=5)
    z = np.zeros_like(y)
    # no l1 term: the TV-l2 chain
    x = _lib.chain_prox_pq(_gpu(y), _gpu(z), alpha=0.0, lam=0.15).cpu().numpy()
    xt = _lib.chain_prox(_gpu(y), lam=0.15).cpu().numpy()
    assert np.abs(x - xt).max() <= TOL
    # no TV: soft threshold towards f
    f = rng.uniform(0, 1, y.shape).astype(np.float32)
    x = _lib.chain_prox_pq(_gpu(y), _gpu(f), alpha=0.2, lam=0.0).cpu().numpy()
    ref = np.where(y + 0.2 < f, y + 0.2, np.where(y - 0.2 > f, y - 0.2, f))
    assert np.abs(x - ref).max() <= 1e-6


def test_overflow_path():
    # a steep ramp with a large TV weight keeps about n/2 breakpoints
    n = 400
    b = np.tile((-np.arange(n) / n).astype(np.float32), (4, 1))
    f = np.tile(np.linspace(0, 1, n, dtype=np.float32), (4, 1))
    ws = _lib.workspace(_lib.load().tv_chain_pq_workspace_size(4, n), DEV, "pq-overflow")
    x = _lib.chain_prox_pq(_gpu(b), _gpu(f), alpha=0.01, lam=n / 16.0, ws=ws).cpu().numpy()
    assert _lib.workspace_status(ws)[1] >= 4
    xr = oracle.chain_solve_pq(np.ones(4 * n), b.ravel(), np.full(4 * n, 0.01), f.ravel(),
                               np.full(4 * n, n / 16.0), np.arange(5) * n)
    assert np.abs(x.ravel() - xr).max() <= TOL


def test_pq_halves_at_full_ring_capacity():
    """Piecewise-quadratic chains whose half messages peak at exactly 16 entries (a
    24-node ramp of b and f with heavy weights, at either end of a 64-node chain; every
    node inserts its own f): the ring of each half wraps all the way round. Against the
    oracle."""
    n = 64
    bs, fs, ws = [], [], []
    for k in range(16):
        rng = np.random.default_rng(60 + k)
        b = np.concatenate([-np.arange(24) / 10.0, rng.uniform(0, 1, n - 24)])
        f = np.concatenate([np.arange(24) / 10.0, rng.uniform(0, 1, n - 24)])
        w = np.concatenate([np.full(24, 5.0), np.full(n - 24, 0.05)])
        if k % 2:  # mirrored: the ramp in the right half
            b, f = b[::-1].copy(), f[::-1].copy()
            w = np.concatenate([w[:n - 1][::-1], [0.0]])
        bs.append(b)
        fs.append(f)
        ws.append(w)
    b = np.concatenate(bs).astype(np.float32)
    f = np.concatenate(fs).astype(np.float32)
    w = np.concatenate(ws).astype(np.float32)
    a = np.ones_like(b)
    al = np.full_like(b, 0.05)
    off = (np.arange(17) * n).astype(np.int64)
    x = _lib.chain_prox_pq(_gpu(b), _gpu(f), alpha=_gpu(al), w=_gpu(w),
                           offsets=torch.from_numpy(off).to(DEV), max_len=n).cpu().numpy()
    xr = oracle.chain_solve_pq(a, b, al, f, w, off)
    assert np.abs(x - xr).max() <= TOL
