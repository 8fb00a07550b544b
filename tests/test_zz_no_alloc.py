"""The allocation-free chain solve, called through the C ABI, against tv_chain_solve
and against the FP64 oracle.

tv_chain_solve_noalloc serves callers that must not call cudaMalloc (for example
code inside a framework that has reserved the GPU's memory for its own caching
allocator); its scratch is a fixed array in device memory shared by all calls.
This file is collected last so that a stop-at-first-failure run has already run
every other test; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
TOL = 2e-5
DEV = "cuda:0"


def _noalloc(y, w=None, lam=0.0, offsets=None, max_len=None):
    lib = _lib.load()
    if offsets is None:
        num_chains, max_len = y.shape
    else:
        num_chains = offsets.numel() - 1
    x = torch.empty_like(y)
    st = lib.tv_chain_solve_noalloc(
        ctypes.c_void_p(y.data_ptr()), None if w is None else ctypes.c_void_p(w.data_ptr()),
        float(lam), None if offsets is None else ctypes.c_void_p(offsets.data_ptr()),
        num_chains, max_len, ctypes.c_void_p(x.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == _lib.TV_OK, lib.tv_last_error()
    return x


def test_noalloc_matches_workspace_entry_point_twice():
    # call 1: a uniform batch (512 chains of 256 nodes, lambda 0.2)
    y1 = torch.from_numpy(synth.chain_batch(512, 256, seed0=0)).to(DEV)
    a1 = _noalloc(y1, lam=0.2)
    b1 = _lib.chain_prox(y1, lam=0.2)
    # call 2, right after: ragged chains with per-edge weights (the shared scratch
    # still holds call 1's records and must not leak into this result)
    lengths = [0, 1, 2, 17, 33, 300, 5, 1000, 64, 129] * 8
    y2n, off = synth.ragged_chain_batch(lengths, seed0=3)
    w2n = np.random.default_rng(1).uniform(0.0, 0.3, size=y2n.shape).astype(np.float32)
    y2 = torch.from_numpy(y2n).to(DEV)
    w2 = torch.from_numpy(w2n).to(DEV)
    offd = torch.from_numpy(off).to(DEV)
    a2 = _noalloc(y2, w2, offsets=offd, max_len=max(lengths))
    b2 = _lib.chain_prox(y2, w2, offsets=offd, max_len=max(lengths))
    torch.cuda.synchronize()
    assert (a1 - b1).abs().max().item() <= TOL
    assert (a2 - b2).abs().max().item() <= TOL
    # both calls element by element against the FP64 oracle
    y1n = y1.cpu().numpy()
    r1 = oracle.chain_solve_batch(y1n.ravel(), np.arange(513, dtype=np.int64) * 256, lam=0.2)
    assert np.abs(a1.cpu().numpy().ravel() - r1).max() <= TOL
    r2 = oracle.chain_solve_batch(y2n, off, w=w2n)
    assert np.abs(a2.cpu().numpy() - r2).max() <= TOL


def test_noalloc_near_its_scratch_limit_against_the_oracle():
    # 640 chains of 1024 nodes: records and reserve take about 15.7 of the 16 MiB, so
    # the records of the last warps sit at the far end of the fixed array
    lib = _lib.load()
    need = lib.tv_chain_workspace_size(640, 1024)
    assert need <= 16 << 20
    yn = synth.chain_batch(640, 1024, seed0=500)
    y = torch.from_numpy(yn).to(DEV)
    for _ in range(2):  # two calls in a row on the same scratch
        x = _noalloc(y, lam=0.15)
        torch.cuda.synchronize()
        r = oracle.chain_solve_batch(yn.ravel(), np.arange(641, dtype=np.int64) * 1024, lam=0.15)
        assert np.abs(x.cpu().numpy().ravel() - r).max() <= TOL


def test_noalloc_rejects_batches_beyond_its_scratch():
    lib = _lib.load()
    # 4096 x 1024 nodes need ~100 MB of scratch: rejected on the host before any
    # launch, so the (never dereferenced) buffer addresses below are only compared.
    y_addr, x_addr = 0x100000000, 0x200000000
    st = lib.tv_chain_solve_noalloc(ctypes.c_void_p(y_addr), None, 0.1, None, 4096, 1024,
                                    ctypes.c_void_p(x_addr), None)
    assert st == _lib.TV_ERR_INVALID
    assert b"scratch" in lib.tv_last_error()
