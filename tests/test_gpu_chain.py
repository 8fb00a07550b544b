"""GPU parity of the batched chain solver against the FP64 oracle (eq. 1D-ROF).

Bar: max |x_gpu - x_oracle| <= 2e-5 on [0, 1]-range data, the FP32 tolerance
the workload targets (the oracle is exact up to FP64 rounding; the kernel runs
the same dynamic program in FP32).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth
from tests import pins

pytestmark = pytest.mark.gpu
TOL = 2e-5
DEV = "cuda:0"


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _rows(y, lam=0.0, w=None):
    return _lib.chain_prox(_gpu(y), None if w is None else _gpu(w), lam=lam).cpu().numpy()


def test_config0_rows_uniform():
    """512 independent chains of length 256 (a 256x256 image's rows and columns), lambda = 0.2."""
    y = synth.chain_batch(512, 256, seed0=0)
    x = _rows(y, lam=0.2)
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(513) * 256, lam=0.2).reshape(y.shape)
    assert np.abs(x - xr).max() <= TOL


def test_config0_as_columns():
    y = synth.chain_batch(512, 256, seed0=0)
    cols = np.ascontiguousarray(y.T)  # (256, 512): chain k is column k
    x = _lib.chain_prox_columns(_gpu(cols), lam=0.2).cpu().numpy()
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(513) * 256, lam=0.2).reshape(y.shape)
    assert np.abs(x.T - xr).max() <= TOL


@pytest.mark.parametrize("layout", ["rows", "cols"])
def test_per_edge_weights(layout):
    rng = np.random.default_rng(3)
    y = synth.chain_batch(96, 203, seed0=40)
    w = rng.uniform(0.0, 0.4, size=y.shape).astype(np.float32)
    w[:, ::17] = 0.0  # decoupled edges
    if layout == "rows":
        x = _rows(y, w=w)
    else:
        x = _lib.chain_prox_columns(_gpu(y.T.copy()), _gpu(w.T.copy())).cpu().numpy().T
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(97) * 203, w=w.ravel()).reshape(y.shape)
    assert np.abs(x - xr).max() <= TOL


def test_ragged_offsets_and_edge_lengths():
    lengths = [0, 1, 2, 3, 15, 16, 17, 31, 32, 33, 1000, 0, 5, 257, 1, 64] * 5 + [1023, 7]
    y, off = synth.ragged_chain_batch(lengths, seed0=11)
    w = np.random.default_rng(4).uniform(0, 0.3, size=y.shape).astype(np.float32)
    for weights in (None, w):
        x = _lib.chain_prox(_gpu(y), None if weights is None else _gpu(weights), lam=0.15,
                            offsets=_gpu(off), max_len=max(lengths)).cpu().numpy()
        xr = oracle.chain_solve_batch(y, off, w=weights, lam=0.15)
        assert np.abs(x - xr).max() <= TOL
    # one-node chains return y exactly
    ones = off[:-1][np.diff(off) == 1]
    np.testing.assert_array_equal(x[ones], y[ones])


def test_overflow_reserve_path():
    """A steep ramp with a weight just under the all-fused threshold keeps about n/2
    breakpoints, more than fit on chip; mixed into warps with ordinary chains."""
    n = 512
    ramp = (-np.arange(n) / n).astype(np.float32)
    y = synth.chain_batch(64, n, seed0=5)
    y[::3] = ramp
    w = np.full(y.shape, 0.05, dtype=np.float32)
    w[::3] = n / 16.0  # the ramp's all-fused threshold is about n/8: ~n/2 breakpoints
    ws = _lib.workspace(_lib.load().tv_chain_workspace_size(64, n), DEV, "overflow-test")
    x = _lib.chain_prox(_gpu(y), _gpu(w), ws=ws).cpu().numpy()
    status, overflowed = _lib.workspace_status(ws)
    assert status == _lib.TV_OK
    assert overflowed >= 20
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(65) * n, w=w.ravel()).reshape(y.shape)
    assert np.abs(x - xr).max() <= TOL


def test_malformed_offsets_are_flagged_not_faulted():
    y = np.zeros(100, np.float32)
    off = np.array([0, 10, 5, 100], np.int64)  # decreasing
    ws = _lib.workspace(_lib.load().tv_chain_workspace_size(3, 100), DEV, "bad-offsets")
    _lib.chain_prox(_gpu(y), lam=0.1, offsets=_gpu(off), max_len=100, ws=ws)
    status, _ = _lib.workspace_status(ws)
    assert status == _lib.TV_ERR_INVALID
    off = np.array([0, 50, 100], np.int64)  # longer than max_len
    _lib.chain_prox(_gpu(y), lam=0.1, offsets=_gpu(off), max_len=20, ws=ws)
    assert _lib.workspace_status(ws)[0] == _lib.TV_ERR_INVALID
    _lib.chain_prox(_gpu(y), lam=0.1, offsets=_gpu(off), max_len=50, ws=ws)
    assert _lib.workspace_status(ws)[0] == _lib.TV_OK


def test_closed_forms_on_gpu():
    y = synth.chain_batch(64, 300, seed0=9)
    np.testing.assert_allclose(_rows(y, lam=0.0), y, atol=1e-6)          # w = 0: x = y
    # a weight above max_k |sum_{j<=k} (mean - y_j)| fuses every edge: x = mean(y).
    # (FP32 breakpoints sit near y +- w, so the error bound scales with |w|; keep w modest.)
    yy = synth.chain_batch(64, 64, seed0=9).astype(np.float64)
    thr = np.abs(np.cumsum(yy.mean(axis=1, keepdims=True) - yy, axis=1)).max()
    big = _rows(yy.astype(np.float32), lam=float(thr) * 1.01)
    np.testing.assert_allclose(big, np.repeat(yy.mean(axis=1)[:, None], 64, 1), atol=TOL)
    const = np.full((32, 100), 0.25, np.float32)
    np.testing.assert_allclose(_rows(const, lam=0.3), const, atol=1e-7)


def test_kkt_certificate_of_gpu_output():
    y = synth.chain_batch(32, 1024, seed0=21)
    x = _rows(y, lam=0.15).astype(np.float64)
    for k in range(32):
        assert pins.kkt_residual(y[k], 0.15, x[k]) < 2e-3  # FP32 rounding of u sums over 1024 nodes


def test_bench_size_sampled():
    """The benchmark's chain workload (65536 chains x 1024, lambda 0.15): sampled chains
    against the oracle, and invariants on every chain."""
    B, n = 65536, 1024
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(B, size=96, replace=False))
    y = np.empty((B, n), np.float32)
    base = synth.chain_batch(256, n, seed0=1000)
    y[:] = np.tile(base, (B // 256, 1))  # 256 distinct chains, repeated
    yg = _gpu(y)
    x = _lib.chain_prox(yg, lam=0.15)
    xs = x[torch.from_numpy(sample).to(DEV)].cpu().numpy()
    xr = oracle.chain_solve_batch(y[sample].ravel(), np.arange(len(sample) + 1) * n, lam=0.15)
    assert np.abs(xs.ravel() - xr).max() <= TOL
    # mean preservation (sum_i x_i = sum_i y_i) on every chain
    d = (x.double().sum(1) - yg.double().sum(1)).abs().max().item()
    assert d < 5e-3
    # identical inputs give identical outputs wherever they sit in the batch
    xv = x.view(B // 256, 256, n)
    assert torch.equal(xv[0], xv[-1])


@pytest.mark.parametrize("B,n", [(65536, 1024), (262144, 256), (16384, 4096)])
def test_sweep_sizes_per_edge_sampled(B, n):
    """The benchmark's per-edge sweep batches (256 distinct chains of the chain workload,
    edge weights U[0.05, 0.3], tiled to B chains; 16-byte staged rows on the default
    path): sampled chains against the oracle, mean preservation on every chain."""
    base = synth.chain_batch(256, n, seed0=2000)
    wrow = np.random.default_rng(3).uniform(0.05, 0.3, size=(256, n)).astype(np.float32)
    yg = _gpu(base).repeat(B // 256, 1)
    wg = _gpu(wrow).repeat(B // 256, 1)
    x = _lib.chain_prox(yg, wg)
    sample = np.sort(np.random.default_rng(1).choice(B, size=48, replace=False))
    xs = x[torch.from_numpy(sample).to(DEV)].cpu().numpy()
    xr = oracle.chain_solve_batch(base[sample % 256].ravel(), np.arange(len(sample) + 1) * n,
                                  w=wrow[sample % 256].ravel())
    assert np.abs(xs.ravel() - xr).max() <= TOL
    d = (x.double().sum(1) - yg.double().sum(1)).abs().max().item()
    assert d < 5e-3


@pytest.mark.parametrize("nc", [2048, 2049, 3000, 4096])
def test_default_path_around_the_warp_kernel_threshold(nc):
    """Batches of 16-byte aligned rows leave the warp-per-chain kernel above 2048 chains
    by default (and other batches above 4096): both sides of that threshold, a ragged
    last warp included, against the oracle on every chain."""
    n = 128
    y = synth.chain_batch(nc, n, seed0=300)
    w = np.random.default_rng(nc).uniform(0.05, 0.3, size=y.shape).astype(np.float32)
    off = np.arange(nc + 1) * n
    x = _rows(y, lam=0.2)
    assert np.abs(x.ravel() - oracle.chain_solve_batch(y.ravel(), off, lam=0.2)).max() <= TOL
    x = _rows(y, w=w)
    assert np.abs(x.ravel() - oracle.chain_solve_batch(y.ravel(), off, w=w.ravel())).max() <= TOL


@pytest.mark.parametrize("split", [0, 1, 2])
def test_middle_rooted_chains(split):
    """Chains solved by one warp from one end (0), rooted at their middle node with the
    two halves in one warp (1, the default for batches solved one chain per warp) or in
    two warps (2): against the oracle, on lengths around the split threshold (64), odd
    and even, and longer than the shared-memory records."""
    lengths = [63, 64, 65, 66, 127, 128, 129, 2, 1, 300, 4097, 5000, 64, 1000]
    y, off = synth.ragged_chain_batch(lengths, seed0=77)
    w = np.random.default_rng(8).uniform(0, 0.3, size=y.shape).astype(np.float32)
    try:
        _lib.set_coop_split(split)
        for weights in (None, w):
            x = _lib.chain_prox(_gpu(y), None if weights is None else _gpu(weights), lam=0.2,
                                offsets=_gpu(off), max_len=max(lengths)).cpu().numpy()
            xr = oracle.chain_solve_batch(y, off, w=weights, lam=0.2)
            assert np.abs(x - xr).max() <= TOL
        # uniform batch as columns
        yc = synth.chain_batch(40, 777, seed0=3)
        xc = _lib.chain_prox_columns(_gpu(yc.T.copy()), lam=0.1).cpu().numpy().T
        xr = oracle.chain_solve_batch(yc.ravel(), np.arange(41) * 777, lam=0.1).reshape(yc.shape)
        assert np.abs(xc - xr).max() <= TOL
    finally:
        _lib.set_coop_split(1)


@pytest.fixture(params=[2, 1, 0], ids=["fixed-shape", "middle-rooted", "one-end"])
def thread_path(request):
    """Every batch on the one-thread-per-chain kernels: chains of 64 nodes or more rooted
    at their middle node with a thread per half, each lane at its own pace (2, the
    default) or with the lanes' updates in step (1), or one thread from one end (0)."""
    _lib.set_coop_max_chains(1)
    _lib.set_thread_split(request.param)
    yield
    _lib.set_coop_max_chains(0)
    _lib.set_thread_split(2)


def test_thread_kernel_rows_columns_weights(thread_path):
    y = synth.chain_batch(512, 256, seed0=0)
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(513) * 256, lam=0.2).reshape(y.shape)
    assert np.abs(_rows(y, lam=0.2) - xr).max() <= TOL
    x = _lib.chain_prox_columns(_gpu(np.ascontiguousarray(y.T)), lam=0.2).cpu().numpy()
    assert np.abs(x.T - xr).max() <= TOL
    rng = np.random.default_rng(3)
    yw = synth.chain_batch(96, 203, seed0=40)
    w = rng.uniform(0.0, 0.4, size=yw.shape).astype(np.float32)
    w[:, ::17] = 0.0
    xw = oracle.chain_solve_batch(yw.ravel(), np.arange(97) * 203, w=w.ravel()).reshape(yw.shape)
    assert np.abs(_rows(yw, w=w) - xw).max() <= TOL
    xc = _lib.chain_prox_columns(_gpu(yw.T.copy()), _gpu(w.T.copy())).cpu().numpy().T
    assert np.abs(xc - xw).max() <= TOL


def test_thread_kernel_ragged_long_and_overflow(thread_path):
    lengths = [0, 1, 2, 3, 15, 16, 17, 31, 32, 33, 1000, 0, 5, 257, 1, 64, 4097, 2048] * 3
    y, off = synth.ragged_chain_batch(lengths, seed0=12)
    w = np.random.default_rng(5).uniform(0, 0.3, size=y.shape).astype(np.float32)
    for weights in (None, w):
        x = _lib.chain_prox(_gpu(y), None if weights is None else _gpu(weights), lam=0.15,
                            offsets=_gpu(off), max_len=max(lengths)).cpu().numpy()
        assert np.abs(x - oracle.chain_solve_batch(y, off, w=weights, lam=0.15)).max() <= TOL
    # a steep ramp keeps ~n/2 breakpoints: more than the ring holds (overflow path)
    n = 512
    yy = synth.chain_batch(64, n, seed0=5)
    yy[::3] = (-np.arange(n) / n).astype(np.float32)
    ww = np.full(yy.shape, 0.05, dtype=np.float32)
    ww[::3] = n / 16.0
    ws = _lib.workspace(_lib.load().tv_chain_workspace_size(64, n), DEV, "overflow-thread")
    x = _lib.chain_prox(_gpu(yy), _gpu(ww), ws=ws).cpu().numpy()
    assert _lib.workspace_status(ws)[1] >= 20
    xr = oracle.chain_solve_batch(yy.ravel(), np.arange(65) * n, w=ww.ravel()).reshape(yy.shape)
    assert np.abs(x - xr).max() <= TOL
    # one weight for every edge on aligned rows (staged 16 bytes at a time): every chain
    # is the ramp, and every one overflows
    yr = np.tile((-np.arange(n) / n).astype(np.float32), (32, 1))
    ws2 = _lib.workspace(_lib.load().tv_chain_workspace_size(32, n), DEV, "overflow-thread-vec")
    x = _lib.chain_prox(_gpu(yr), lam=n / 16.0, ws=ws2).cpu().numpy()
    assert _lib.workspace_status(ws2)[1] >= 1
    xr = oracle.chain_solve_batch(yr.ravel(), np.arange(33) * n, lam=n / 16.0).reshape(yr.shape)
    assert np.abs(x - xr).max() <= TOL


def test_thread_kernel_aligned_rows_stay_in_bounds(thread_path):
    """Uniform chains whose arrays are 16-byte aligned with a length a multiple of 4 are
    staged and stored 16 bytes at a time per half. The lengths here end a half inside a
    4-node group or an 8-node chunk. The output sits in a larger buffer whose guard
    entries must stay NaN. A pointer one float off the 16-byte grid takes the
    node-by-node path."""
    rng = np.random.default_rng(8)
    for n in (64, 68, 72, 100, 132, 260):
        B = 40
        y = synth.chain_batch(B, n, seed0=n)
        w = rng.uniform(0.0, 0.4, size=y.shape).astype(np.float32)
        for weights in (None, w):
            xr = oracle.chain_solve_batch(y.ravel(), np.arange(B + 1) * n,
                                          w=None if weights is None else weights.ravel(),
                                          lam=0.15).reshape(y.shape)
            buf = torch.full((B * n + 8,), float("nan"), device=DEV)
            out = buf[4:4 + B * n].view(B, n)
            _lib.chain_prox(_gpu(y), None if weights is None else _gpu(weights), lam=0.15, out=out)
            g = buf.cpu().numpy()
            assert np.isnan(g[:4]).all() and np.isnan(g[4 + B * n:]).all(), n
            assert np.abs(g[4:4 + B * n].reshape(B, n) - xr).max() <= TOL, n
            yo = torch.empty(B * n + 1, device=DEV)[1:].view(B, n)
            yo.copy_(_gpu(y))
            xo = _lib.chain_prox(yo, None if weights is None else _gpu(weights), lam=0.15)
            assert np.abs(xo.cpu().numpy() - xr).max() <= TOL, n


def test_thread_kernel_closed_forms(thread_path):
    y = synth.chain_batch(64, 300, seed0=9)
    np.testing.assert_allclose(_rows(y, lam=0.0), y, atol=1e-6)
    yy = synth.chain_batch(64, 64, seed0=9).astype(np.float64)
    thr = np.abs(np.cumsum(yy.mean(axis=1, keepdims=True) - yy, axis=1)).max()
    big = _rows(yy.astype(np.float32), lam=float(thr) * 1.01)
    np.testing.assert_allclose(big, np.repeat(yy.mean(axis=1)[:, None], 64, 1), atol=TOL)
    x = _rows(synth.chain_batch(32, 1024, seed0=21), lam=0.15).astype(np.float64)
    yk = synth.chain_batch(32, 1024, seed0=21)
    for k in range(32):
        assert pins.kkt_residual(yk[k], 0.15, x[k]) < 2e-3


def test_halves_at_full_ring_capacity():
    """Chains whose half messages peak at exactly 16 breakpoints, all the lanes of a
    16-lane half (a 28-node steep ramp with heavy weights, at the start of the chain or,
    mirrored, at its end): the ring of each half wraps all the way round without falling
    back to the whole warp. Against the oracle."""
    n = 80
    ys, ws = [], []
    for k in range(16):
        base = np.concatenate([(-np.arange(28) / 40.0),
                               np.random.default_rng(k).uniform(0, 1, n - 28)])
        w = np.concatenate([np.full(28, 2.5), np.full(n - 28, 0.05)])
        if k % 2:  # mirrored: the ramp in the right half (edge i of the mirror is n-2-i)
            base = base[::-1].copy()
            w = np.concatenate([w[:n - 1][::-1], [0.0]])
        ys.append(base)
        ws.append(w)
    y = np.stack(ys).astype(np.float32)
    w = np.stack(ws).astype(np.float32)
    ws_ = _lib.workspace(_lib.load().tv_chain_workspace_size(16, n), DEV, "full-ring")
    x = _lib.chain_prox(_gpu(y), _gpu(w), ws=ws_).cpu().numpy()
    assert _lib.workspace_status(ws_)[1] == 0
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(17) * n, w=w.ravel()).reshape(y.shape)
    assert np.abs(x - xr).max() <= TOL


def test_half_overflow_falls_back_to_the_whole_warp():
    """A chain whose left half needs ~22 breakpoints: more than a 16-lane half holds, fewer
    than the 32 lanes of the whole warp, which solves it without the lane-0 path."""
    n = 80
    base = np.concatenate([(-np.arange(40) / 40.0), np.random.default_rng(0).uniform(0, 1, 40)])
    y = np.tile(base.astype(np.float32), (16, 1))
    w = np.tile(np.concatenate([np.full(40, 2.5), np.full(40, 0.05)]).astype(np.float32), (16, 1))
    ws = _lib.workspace(_lib.load().tv_chain_workspace_size(16, n), DEV, "half-overflow")
    x = _lib.chain_prox(_gpu(y), _gpu(w), ws=ws).cpu().numpy()
    assert _lib.workspace_status(ws)[1] == 0  # never reached the lane-0 path
    xr = oracle.chain_solve_batch(y.ravel(), np.arange(17) * n, w=w.ravel()).reshape(y.shape)
    assert np.abs(x - xr).max() <= TOL
