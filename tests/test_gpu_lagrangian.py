"""GPU parity of the symmetric Lagrangian ROF solver (Sec. 6 split) against the oracle."""
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


@pytest.mark.parametrize("edge_aware", [False, True])
@pytest.mark.parametrize("k", [1, 4, 15])
def test_fixed_iterations_against_oracle(edge_aware, k):
    _, f = synth.shapes_image(96, 130, seed=6, n_shapes=30)
    lam = 0.12
    wh = wv = None
    if edge_aware:
        wh, wv = synth.edge_aware_weights(f, lam)
    x, it, gap, ok = _lib.tv2d_denoise_lagrangian(_gpu(f), lam=lam, w_h=_gpu(wh), w_v=_gpu(wv),
                                                  tau0=10.0, max_iters=k, tol=0.0, check_every=k)
    xo, ito, tro, oko = oracle.tv2d_lagrangian(f, lam=lam, w_h=wh, w_v=wv, tau0=10.0, max_iters=k,
                                               tol=0.0, check_every=k)
    assert it == ito == k
    assert np.abs(x.cpu().numpy() - xo).max() <= TOL
    assert abs(gap - tro[-1]) <= 1e-6 + 1e-3 * abs(tro[-1])


def test_stops_at_the_gap_tolerance():
    _, f = synth.shapes_image(128, 96, seed=8, n_shapes=40)
    x, it, gap, ok = _lib.tv2d_denoise_lagrangian(_gpu(f), lam=0.1, tau0=10.0, max_iters=300,
                                                  tol=1e-4, check_every=5)
    assert ok and gap <= 1e-4 and it % 5 == 0
    xo, ito, tro, oko = oracle.tv2d_lagrangian(f, lam=0.1, tau0=10.0, max_iters=it, tol=0.0,
                                               check_every=it)
    assert np.abs(x.cpu().numpy() - xo).max() <= TOL
    # the same minimiser as the accelerated form, within what the two gaps allow
    xp, itp, gp, okp = _lib.tv2d_denoise(_gpu(f), lam=0.1, max_iters=200, tol=1e-4)
    N = f.size
    assert np.sum((x.cpu().numpy() - xp.cpu().numpy()) ** 2) <= 4 * 2 * 1e-4 * N


def test_no_regulariser_is_the_identity():
    _, f = synth.shapes_image(40, 33, seed=9, n_shapes=10)
    x, it, gap, ok = _lib.tv2d_denoise_lagrangian(_gpu(f), lam=0.0, tau0=10.0, max_iters=3, tol=0.0,
                                                  check_every=1)
    np.testing.assert_allclose(x.cpu().numpy(), f, atol=1e-6)
    assert abs(gap) <= 1e-6


@pytest.mark.parametrize("which", ["h", "v"])
def test_weights_in_one_direction_only(which):
    """Row and column chains run in one launch; here one of them has edge weights and the
    other the uniform lambda."""
    _, f = synth.shapes_image(72, 110, seed=12, n_shapes=25)
    lam = 0.1
    wh, wv = synth.edge_aware_weights(f, lam)
    if which == "h":
        wv = None
    else:
        wh = None
    x, it, gap, ok = _lib.tv2d_denoise_lagrangian(_gpu(f), lam=lam, w_h=_gpu(wh), w_v=_gpu(wv),
                                                  tau0=10.0, max_iters=4, tol=0.0, check_every=4)
    xo, ito, tro, oko = oracle.tv2d_lagrangian(f, lam=lam, w_h=wh, w_v=wv, tau0=10.0, max_iters=4,
                                               tol=0.0, check_every=4)
    assert np.abs(x.cpu().numpy() - xo).max() <= TOL
    assert abs(gap - tro[-1]) <= 1e-6 + 1e-3 * abs(tro[-1])


def test_long_rows_keep_their_records_in_the_workspace():
    """Rows of 5000 nodes: more than a warp keeps in shared memory, so the records of
    every chain of the launch (40 rows and 5000 columns) live in the workspace."""
    _, f = synth.shapes_image(40, 5000, seed=13, n_shapes=60)
    x, it, gap, ok = _lib.tv2d_denoise_lagrangian(_gpu(f), lam=0.1, tau0=10.0, max_iters=2,
                                                  tol=0.0, check_every=2)
    xo, ito, tro, oko = oracle.tv2d_lagrangian(f, lam=0.1, tau0=10.0, max_iters=2, tol=0.0,
                                               check_every=2)
    assert np.abs(x.cpu().numpy() - xo).max() <= TOL


def test_programmatic_launch_gives_identical_results():
    """Kernels launched with a programmatic dependency on their predecessor give
    bitwise the same result as plain stream order."""
    _, f = synth.shapes_image(120, 90, seed=14, n_shapes=30)
    out = {}
    try:
        for on in (True, False):
            _lib.set_programmatic_launch(on)
            x, it, gap, ok = _lib.tv2d_denoise_lagrangian(_gpu(f), lam=0.1, tau0=10.0, max_iters=10,
                                                          tol=0.0, check_every=5)
            out[on] = (x.cpu().numpy(), it, gap)
    finally:
        _lib.set_programmatic_launch(True)
    assert out[True][1] == out[False][1] and out[True][2] == out[False][2]
    assert np.array_equal(out[True][0], out[False][0])
