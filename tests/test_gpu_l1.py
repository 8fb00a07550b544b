"""GPU parity of 2D TV-l1 denoising (Sec. 6: column chains for the dual, row chains with
piecewise-quadratic unaries for the primal) against the oracle's FP64 iteration."""
import numpy as np
import pytest
import torch

import oracle
from paper_1502_07770_gb300 import _lib, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 2e-5
TAU = 0.3


def _gpu(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(DEV)


def _energy(x, f, lam, wh, wv):
    x = x.astype(np.float64)
    f = f.astype(np.float64)
    wh = np.full((x.shape[0], x.shape[1] - 1), lam) if wh is None else wh.astype(np.float64)
    wv = np.full((x.shape[0] - 1, x.shape[1]), lam) if wv is None else wv.astype(np.float64)
    return (np.abs(x - f).sum() + (wh * np.abs(np.diff(x, axis=1))).sum()
            + (wv * np.abs(np.diff(x, axis=0))).sum())


@pytest.mark.parametrize("edge_aware", [False, True])
@pytest.mark.parametrize("k", [1, 5, 25])
def test_fixed_iterations_against_oracle(edge_aware, k):
    f = synth.salt_pepper_image(96, 130, 3)
    lam = 0.35
    wh = wv = None
    if edge_aware:
        wh, wv = synth.edge_aware_weights(f, lam)
    x, it, e, ok = _lib.tv2d_denoise_l1(_gpu(f), lam=lam, w_h=_gpu(wh), w_v=_gpu(wv), tau=TAU,
                                        max_iters=k, tol=0.0, check_every=k)
    xo, eo = oracle.tv2d_l1(f, lam=lam, w_h=wh, w_v=wv, tau=TAU, iters=k)
    assert ok and it == k
    xg = x.cpu().numpy()
    assert np.abs(xg - xo).max() <= TOL
    assert abs(e - eo[-1]) <= 1e-5 * eo[-1]
    # the device energy is the energy of the returned image
    assert abs(e - _energy(xg, f, lam, wh, wv)) <= 1e-5 * e


@pytest.mark.parametrize("shape", [(1, 77), (77, 1), (3, 2), (1, 1), (65, 64), (33, 200)])
def test_ragged_and_degenerate_shapes(shape):
    H, W = shape
    f = np.random.default_rng(H * 1000 + W).uniform(size=shape).astype(np.float32)
    x, it, e, ok = _lib.tv2d_denoise_l1(_gpu(f), lam=0.4, tau=TAU, max_iters=12, tol=0.0,
                                        check_every=4)
    xo, eo = oracle.tv2d_l1(f, lam=0.4, tau=TAU, iters=12)
    assert it == 12
    assert np.abs(x.cpu().numpy() - xo).max() <= TOL
    assert abs(e - eo[-1]) <= 1e-5 * max(eo[-1], 1e-3)


def test_larger_image_several_tiles():
    f = synth.salt_pepper_image(512, 768, 11)
    x, it, e, ok = _lib.tv2d_denoise_l1(_gpu(f), lam=0.5, tau=TAU, max_iters=10, tol=0.0,
                                        check_every=10)
    xo, eo = oracle.tv2d_l1(f, lam=0.5, tau=TAU, iters=10)
    assert np.abs(x.cpu().numpy() - xo).max() <= TOL
    assert abs(e - eo[-1]) <= 1e-5 * eo[-1]


def test_stops_at_the_energy_tolerance():
    f = synth.salt_pepper_image(64, 90, 5)
    x, it, e, ok = _lib.tv2d_denoise_l1(_gpu(f), lam=0.3, tau=TAU, max_iters=2000, tol=1e-6,
                                        check_every=20)
    assert ok and it % 20 == 0 and it < 2000
    xo, eo = oracle.tv2d_l1(f, lam=0.3, tau=TAU, iters=it)
    assert abs(e - eo[-1]) <= 1e-5 * eo[-1]
    # stopped because two checks agreed, and the oracle's energies agree there too
    assert abs(eo[-1] - eo[-21]) <= 1e-5 * eo[-1]


def test_no_regulariser_is_the_identity():
    f = synth.salt_pepper_image(40, 33, 9)
    x, it, e, ok = _lib.tv2d_denoise_l1(_gpu(f), lam=0.0, tau=TAU, max_iters=3, tol=0.0,
                                        check_every=1)
    np.testing.assert_allclose(x.cpu().numpy(), f, atol=1e-6)
    assert abs(e) <= 1e-5


def test_invalid_arguments():
    f = _gpu(np.zeros((8, 8)))
    for kw in ({"tau": 0.0}, {"tau": float("inf")}, {"max_iters": 0}, {"check_every": 0},
               {"lam": -1.0}, {"tol": -1.0}):
        args = dict(lam=0.1, tau=TAU, max_iters=5, tol=0.0, check_every=1)
        args.update(kw)
        with pytest.raises(_lib.TVError):
            _lib.tv2d_denoise_l1(f, **args)


def test_programmatic_launch_gives_identical_results():
    """The TV-l1 solver's kernels launched with a programmatic dependency on their
    predecessor give bitwise the same iterate, iteration count and energy as plain
    stream order."""
    f = synth.salt_pepper_image(200, 260, seed=21)
    out = {}
    try:
        for on in (True, False):
            _lib.set_programmatic_launch(on)
            x, it, e, ok = _lib.tv2d_denoise_l1(_gpu(f), lam=0.5, tau=TAU, max_iters=20, tol=0.0,
                                                check_every=5)
            out[on] = (x.cpu().numpy(), it, e)
    finally:
        _lib.set_programmatic_launch(True)
    assert out[True][1] == out[False][1] and out[True][2] == out[False][2]
    assert np.array_equal(out[True][0], out[False][0])
