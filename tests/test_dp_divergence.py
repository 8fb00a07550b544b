"""The host replay of the thread-form chain update (used for its loop statistics) solves
the chain: its records and the backward clips of Algorithm 2 give the oracle's minimiser."""
import numpy as np

import oracle
from paper_1502_07770_gb300 import synth
from tests import dp_divergence as dd


def test_replay_solves_the_chain():
    y = synth.chain_batch(12, 300, seed0=50)
    for k in range(12):
        x = dd.replay_chain(y[k], 0.15)
        xo = oracle.chain_solve_batch(y[k], np.array([0, 300]), lam=0.15)
        assert np.abs(x - xo).max() <= 2e-5


def test_statistics_are_consistent():
    y = synth.chain_batch(16, 256, seed0=1000)
    r = dd.warp_stats(y, 0.15)
    assert np.all(r["lane_mean"] >= 0)
    assert np.all(r["warp_max"] >= r["lane_mean"])  # a warp runs at least its mean lane
    assert 2 <= r["size_max"] <= 16
