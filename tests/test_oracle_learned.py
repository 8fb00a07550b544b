"""Pins of the FP64 reference of the warm-start network (no GPU)."""
import numpy as np
import torch

from oracle import learned


def test_delta_kernel_is_a_shift():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 16))
    w = np.zeros((16, 3, 3, 16))
    for c in range(16):
        w[c, 0, 2, c] = 1.0  # tap (ky=0, kx=2): input at (y-1, x+1)
    out = learned.conv3x3(x, w).numpy()
    ref = np.zeros_like(x)
    ref[:, 1:, :-1, :] = x[:, :-1, 1:, :]
    np.testing.assert_array_equal(out, ref)


def test_head_is_the_adjoint_of_the_vertical_difference():
    rng = np.random.default_rng(1)
    o = rng.normal(size=(3, 6, 5))
    lam = np.array([0.1, 0.2, 0.3])
    y = learned.dual_head(o, lam).numpy()
    p = lam[:, None, None] * np.tanh(o)
    p[:, -1] = 0.0
    x = rng.normal(size=(3, 6, 5))
    dvx = np.zeros_like(x)
    dvx[:, :-1] = x[:, 1:] - x[:, :-1]  # D_v x on vertical edges
    assert abs((y * x).sum() - (p * dvx).sum()) < 1e-12  # <D_v^T p, x> = <p, D_v x>
    assert np.all(np.abs(p) <= lam[:, None, None])       # dual feasible


def test_gradients_against_finite_differences():
    rng = np.random.default_rng(2)
    shapes = [(32, 16), (32, 32), (32, 32), (16, 32)]
    params = [(rng.normal(scale=0.1, size=(co, 3, 3, ci)), rng.normal(scale=0.05, size=co))
              for co, ci in shapes]
    f = rng.uniform(size=(1, 5, 6))
    lam = np.array([0.2])
    t = rng.normal(scale=0.05, size=(1, 5, 6))
    loss, grads, _ = learned.loss_and_grads(params, f, lam, t)
    h = 1e-6
    for li, idx in ((0, (3, 1, 2, 0)), (1, (5, 0, 0, 7)), (3, (0, 2, 1, 4))):
        wp = [(w.copy(), b.copy()) for w, b in params]
        wm = [(w.copy(), b.copy()) for w, b in params]
        wp[li][0][idx] += h
        wm[li][0][idx] -= h
        lp = learned.loss_and_grads(wp, f, lam, t)[0]
        lm = learned.loss_and_grads(wm, f, lam, t)[0]
        assert abs((lp - lm) / (2 * h) - grads[li][0][idx]) < 1e-6
    bp = [(w.copy(), b.copy()) for w, b in params]
    bp[2][1][3] += h
    bm = [(w.copy(), b.copy()) for w, b in params]
    bm[2][1][3] -= h
    fd = (learned.loss_and_grads(bp, f, lam, t)[0] - learned.loss_and_grads(bm, f, lam, t)[0]) / (2 * h)
    assert abs(fd - grads[2][1][3]) < 1e-6


def test_first_adam_step_moves_by_lr_times_sign():
    # at step 1 the bias-corrected moments are g and g^2, so the move is lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, -7.0])
    w, m, v = learned.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 0.01, 0.9, 0.999, 0.0, 1)
    np.testing.assert_allclose(w, -0.01 * np.sign(g), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_head_gradient_against_finite_differences():
    rng = np.random.default_rng(4)
    o = rng.normal(size=(2, 5, 4))
    lam = np.array([0.15, 0.25])
    t = rng.normal(scale=0.1, size=(2, 5, 4))
    _, loss, g = learned.head_loss_grad(o, lam, t)
    h = 1e-6
    for idx in ((0, 0, 0), (1, 3, 2), (0, 4, 1)):
        op, om = o.copy(), o.copy()
        op[idx] += h
        om[idx] -= h
        fd = (learned.head_loss_grad(op, lam, t)[1] - learned.head_loss_grad(om, lam, t)[1]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8
    assert np.all(g[:, -1] == 0.0)  # the last row has no vertical edge


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(5)
    x = rng.normal(size=(2, 6, 7, 16))
    w = rng.normal(size=(32, 3, 3, 16))
    dy = rng.normal(size=(2, 6, 7, 32))
    dx, dw, db = learned.conv3x3_grads(x, w, dy)
    # <conv(x), dy> = <x, dx> (linearity in x), = <w, dw> (linearity in w)
    lhs = float((learned.conv3x3(x, w).numpy() * dy).sum())
    assert abs(lhs - (x * dx).sum()) < 1e-9 * abs(lhs) + 1e-9
    assert abs(lhs - (w * dw).sum()) < 1e-9 * abs(lhs) + 1e-9
    np.testing.assert_allclose(db, dy.sum(axis=(0, 1, 2)))


def test_bf16_storage_variant_reduces_to_plain_on_bf16_exact_data():
    # with inputs, weights and every stored tensor exactly representable in bfloat16 the two
    # reference variants agree; pick data where that holds: zero hidden weights make every
    # activation the (bf16-exact) bias ReLU
    shapes = [(32, 16), (32, 32), (32, 32), (16, 32)]
    params = [(np.zeros((co, 3, 3, ci)), np.full(co, 0.25)) for co, ci in shapes]
    f = np.full((1, 4, 5), 0.5)
    lam = np.array([0.125])
    t = np.zeros((1, 4, 5))
    l1, g1, y1 = learned.loss_and_grads(params, f, lam, t)
    l2, g2, y2 = learned.loss_and_grads_bf16_storage(params, f, lam, t)
    assert l1 == l2
    np.testing.assert_array_equal(y1, y2)
