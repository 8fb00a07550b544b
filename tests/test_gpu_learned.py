"""GPU parity of the warm-start network kernels against the FP64 CPU reference.

Sizes are ragged against the 8 x 16 output tile (H = 13, W = 37) so that partial
tiles, image borders and several tiles per image are all covered. Inputs are
BF16; the reference computes in float64 on the same BF16 values, so the only
differences are FP32 accumulation order and the BF16 rounding of BF16 outputs.
"""
import numpy as np
import pytest
import torch

from oracle import learned as ref
from paper_1502_07770_gb300 import _lib, learned, synth

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
B, H, W = 2, 13, 37
PAIRS = [(16, 32), (32, 32), (32, 16), (16, 16)]


def _bf16(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(*shape, generator=g) * scale).to(torch.bfloat16).to(DEV)


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _vp(t):
    return learned._vp(t)


def _stream():
    return _lib._stream(torch.device(DEV))


def _ws(b=B, h=H, w=W):
    n = _lib.load().tv_net_workspace_size(b, h, w)
    assert n > 0
    return torch.empty(n, dtype=torch.uint8, device=DEV)


def _bf16_close(got, want, rel=2.0 ** -8, atol=1e-5):
    err = np.abs(got - want)
    assert np.all(err <= rel * np.abs(want) + atol), err.max()


@pytest.mark.parametrize("cin,cout", PAIRS)
def test_conv_forward(cin, cout):
    lib = _lib.load()
    x = _bf16((B, H, W, cin), 1)
    w = _bf16((cout, 3, 3, cin), 2, scale=0.2)
    b = torch.randn(cout, generator=torch.Generator().manual_seed(3)).to(DEV)
    pre = torch.empty(B, H, W, cout, device=DEV)
    act = torch.empty(B, H, W, cout, dtype=torch.bfloat16, device=DEV)
    _lib._check(lib.tv_net_conv3x3(_vp(x), B, H, W, cin, _vp(w), _vp(b), cout, 1, _vp(pre),
                                   _vp(act), _stream()))
    want = ref.conv3x3(_np(x), _np(w), b.cpu().numpy().astype(np.float64)).numpy()
    np.testing.assert_allclose(pre.cpu().numpy(), want, rtol=0, atol=2e-5 * max(1.0, np.abs(want).max()))
    _bf16_close(_np(act), np.maximum(want, 0.0), atol=1e-4)
    # without an activation output, and without bias
    pre2 = torch.empty_like(pre)
    _lib._check(lib.tv_net_conv3x3(_vp(x), B, H, W, cin, _vp(w), None, cout, 0, _vp(pre2), None,
                                   _stream()))
    want2 = ref.conv3x3(_np(x), _np(w)).numpy()
    np.testing.assert_allclose(pre2.cpu().numpy(), want2, rtol=0, atol=2e-5 * max(1.0, np.abs(want2).max()))


@pytest.mark.parametrize("cin,cout", PAIRS)
@pytest.mark.parametrize("shape", [(2, 13, 37), (1, 7, 300), (3, 2, 128)])
def test_conv_forward_tensor_paths(cin, cout, shape):
    """The two tcgen05 forwards (128-pixel row tiles, TMEM accumulators; the second fed
    by TMA with warp roles) and the mma.sync forward against the FP64 reference, on rows
    of one, several and partial tiles, images shorter than the three staged rows, and
    batches of images (TMA zero-fills outside each image)."""
    lib = _lib.load()
    b_, h_, w_ = shape
    x = _bf16((b_, h_, w_, cin), 11)
    w = _bf16((cout, 3, 3, cin), 12, scale=0.2)
    b = torch.randn(cout, generator=torch.Generator().manual_seed(13)).to(DEV)
    want = ref.conv3x3(_np(x), _np(w), b.cpu().numpy().astype(np.float64)).numpy()
    tol = 2e-5 * max(1.0, np.abs(want).max())
    outs = []
    try:
        t0 = lib.tv_net_tensor_timeouts()
        for mode in (2, 1, 0):
            _lib.set_net_tensor_path(mode)
            pre = torch.full((b_, h_, w_, cout), float("nan"), device=DEV)
            act = torch.empty(b_, h_, w_, cout, dtype=torch.bfloat16, device=DEV)
            _lib._check(lib.tv_net_conv3x3(_vp(x), b_, h_, w_, cin, _vp(w), _vp(b), cout, 1,
                                           _vp(pre), _vp(act), _stream()))
            got = pre.cpu().numpy()
            np.testing.assert_allclose(got, want, rtol=0, atol=tol)
            _bf16_close(_np(act), np.maximum(want, 0.0), atol=1e-4)
            outs.append(got)
        assert lib.tv_net_tensor_timeouts() == t0
    finally:
        _lib.set_net_tensor_path(0)
    for o in outs[:-1]:
        np.testing.assert_allclose(o, outs[-1], rtol=0, atol=tol)


def _grouped(x):
    """NHWC (B, H, W, C) -> the channel-group layout (B, H, C/8, W, 8)."""
    b_, h_, w_, c = x.shape
    return x.reshape(b_, h_, w_, c // 8, 8).permute(0, 1, 3, 2, 4).contiguous()


def _ungrouped(x):
    b_, h_, g, w_, _ = x.shape
    return x.permute(0, 1, 3, 2, 4).reshape(b_, h_, w_, g * 8)


@pytest.mark.parametrize("cin,cout", PAIRS)
@pytest.mark.parametrize("shape", [(2, 13, 37), (1, 7, 300), (3, 2, 128), (1, 1, 1)])
def test_conv_forward_grouped_layout(cin, cout, shape):
    """The convolution on the channel-group layout (TMA boxes of whole row runs)
    against the FP64 reference: FP32 pre-activation (NHWC) and the BF16 activation
    (grouped), with and without bias and ReLU, and no timed-out wait."""
    lib = _lib.load()
    b_, h_, w_ = shape
    x = _bf16((b_, h_, w_, cin), 21)
    w = _bf16((cout, 3, 3, cin), 22, scale=0.2)
    b = torch.randn(cout, generator=torch.Generator().manual_seed(23)).to(DEV)
    xg = _grouped(x)
    t0 = lib.tv_net_tensor_timeouts()
    for bias, relu in ((b, 1), (None, 0)):
        want = ref.conv3x3(_np(x), _np(w), None if bias is None else
                           bias.cpu().numpy().astype(np.float64)).numpy()
        tol = 2e-5 * max(1.0, np.abs(want).max())
        pre = torch.full((b_, h_, w_, cout), float("nan"), device=DEV)
        act = torch.full((b_, h_, cout // 8, w_, 8), float("nan"), dtype=torch.bfloat16, device=DEV)
        _lib._check(lib.tv_net_conv3x3_grouped(_vp(xg), b_, h_, w_, cin, _vp(w),
                                               None if bias is None else _vp(bias), cout, relu,
                                               _vp(pre), _vp(act), _stream()))
        np.testing.assert_allclose(pre.cpu().numpy(), want, rtol=0, atol=tol)
        _bf16_close(_np(_ungrouped(act)), np.maximum(want, 0.0) if relu else want, atol=1e-4)
    assert lib.tv_net_tensor_timeouts() == t0


@pytest.mark.parametrize("shape", [(2, 13, 37), (1, 7, 300), (3, 2, 128), (1, 1, 1)])
def test_first_layer_from_the_image(shape):
    """The first layer on tcgen05 with the image rows built in shared memory (f and its
    lambda rounded to BF16, channels 2..15 zero) against the FP64 reference on the packed
    input; the activation comes out in the channel-group layout."""
    lib = _lib.load()
    b_, h_, w_ = shape
    f = torch.rand(b_, h_, w_, generator=torch.Generator().manual_seed(31)).to(DEV)
    lam = torch.tensor([0.05 + 0.1 * i for i in range(b_)], dtype=torch.float32, device=DEV)
    w = _bf16((32, 3, 3, 16), 32, scale=0.3)
    bias = torch.randn(32, generator=torch.Generator().manual_seed(33)).to(DEV)
    act = torch.full((b_, h_, 4, w_, 8), float("nan"), dtype=torch.bfloat16, device=DEV)
    t0 = lib.tv_net_tensor_timeouts()
    _lib._check(lib.tv_net_first_layer(_vp(f), b_, h_, w_, _vp(lam), _vp(w), _vp(bias), _vp(act), 1,
                                       _stream()))
    x = ref.pack_input(_np(f.to(torch.bfloat16)), lam.to(torch.bfloat16).float().cpu().numpy())
    want = ref.conv3x3(x, _np(w), bias.cpu().numpy().astype(np.float64)).numpy()
    _bf16_close(_np(_ungrouped(act)), np.maximum(want, 0.0), atol=1e-4)
    assert lib.tv_net_tensor_timeouts() == t0


@pytest.mark.parametrize("cin", [32, 16])
@pytest.mark.parametrize("shape", [(2, 13, 37), (1, 7, 300), (3, 2, 128), (1, 1, 1)])
def test_last_layer_fused_with_the_dual_head(cin, shape):
    """The last convolution (cin -> 16, grouped input) whose epilogue keeps channel 0 and
    writes p = lambda tanh(o) on the vertical edges, then y = D_v^T p, against the FP64
    reference convolution followed by the reference head."""
    lib = _lib.load()
    b_, h_, w_ = shape
    x = _bf16((b_, h_, w_, cin), 41)
    w = _bf16((16, 3, 3, cin), 42, scale=0.2)
    bias = torch.randn(16, generator=torch.Generator().manual_seed(43)).to(DEV)
    lam = torch.tensor([0.1 + 0.07 * i for i in range(b_)], dtype=torch.float32, device=DEV)
    p = torch.full((b_, h_, w_), float("nan"), device=DEV)
    y = torch.full((b_, h_, w_), float("nan"), device=DEV)
    t0 = lib.tv_net_tensor_timeouts()
    _lib._check(lib.tv_net_conv3x3_dual_head(_vp(_grouped(x)), b_, h_, w_, cin, _vp(w), _vp(bias),
                                             _vp(lam), _vp(p), _vp(y), _stream()))
    o = ref.conv3x3(_np(x), _np(w), bias.cpu().numpy().astype(np.float64))[..., 0]
    lam64 = lam.cpu().numpy().astype(np.float64)
    want_y = ref.dual_head(o, lam64).numpy()
    # |d tanh| <= 1: an FP32-sum difference in o moves y by at most lambda times as much
    tol = 2e-5 * max(1.0, float(o.abs().max())) * float(lam64.max()) * 2 + 1e-6
    np.testing.assert_allclose(y.cpu().numpy(), want_y, rtol=0, atol=tol)
    want_p = lam64[:, None, None] * np.tanh(o.numpy())
    want_p[:, -1] = 0.0
    np.testing.assert_allclose(p.cpu().numpy(), want_p, rtol=0, atol=tol)
    assert lib.tv_net_tensor_timeouts() == t0


@pytest.mark.parametrize("cin,cout", PAIRS)
def test_conv_backward_data_and_weight(cin, cout):
    lib = _lib.load()
    x = _bf16((B, H, W, cin), 4)
    w = _bf16((cout, 3, 3, cin), 5, scale=0.2)
    dy = _bf16((B, H, W, cout), 6)
    mask = torch.randn(B, H, W, cin, generator=torch.Generator().manual_seed(7)).to(DEV)
    dx = torch.empty(B, H, W, cin, dtype=torch.bfloat16, device=DEV)
    flip = torch.empty(32 * 9 * 32, dtype=torch.bfloat16, device=DEV)
    _lib._check(lib.tv_net_conv3x3_backward_data(_vp(dy), B, H, W, cout, _vp(w), cin, _vp(mask),
                                                 _vp(dx), _vp(flip), _stream()))
    dw = torch.zeros(cout, 3, 3, cin, device=DEV)
    db = torch.zeros(cout, device=DEV)
    ws = _ws()
    _lib._check(lib.tv_net_conv3x3_backward_weight(_vp(x), _vp(dy), B, H, W, cin, cout, _vp(dw),
                                                   _vp(db), _vp(ws), ws.numel(), _stream()))
    rdx, rdw, rdb = ref.conv3x3_grads(_np(x), _np(w), _np(dy))
    rdx = rdx * (mask.cpu().numpy() > 0)
    _bf16_close(_np(dx), rdx, atol=1e-4)
    scale = np.abs(rdw).max()
    np.testing.assert_allclose(dw.cpu().numpy(), rdw, rtol=0, atol=2e-5 * scale)
    np.testing.assert_allclose(db.cpu().numpy(), rdb, rtol=0, atol=2e-5 * np.abs(rdb).max())


def test_weight_gradient_accumulates():
    lib = _lib.load()
    x = _bf16((B, H, W, 32), 8)
    dy = _bf16((B, H, W, 32), 9)
    dw = torch.zeros(32, 3, 3, 32, device=DEV)
    ws = _ws()
    for _ in range(2):
        _lib._check(lib.tv_net_conv3x3_backward_weight(_vp(x), _vp(dy), B, H, W, 32, 32, _vp(dw),
                                                       None, _vp(ws), ws.numel(), _stream()))
    again = torch.zeros_like(dw)
    for _ in range(2):
        _lib._check(lib.tv_net_conv3x3_backward_weight(_vp(x), _vp(dy), B, H, W, 32, 32,
                                                       _vp(again), None, _vp(ws), ws.numel(),
                                                       _stream()))
    assert torch.equal(again, dw)  # fixed-order reduction: bitwise reproducible
    _, rdw, _ = ref.conv3x3_grads(_np(x), np.zeros((32, 3, 3, 32)), _np(dy))
    np.testing.assert_allclose(dw.cpu().numpy(), 2 * rdw, rtol=0, atol=4e-5 * np.abs(rdw).max())


def test_head_and_its_gradient():
    lib = _lib.load()
    g = torch.Generator().manual_seed(10)
    o = torch.randn(B, H, W, 16, generator=g).to(DEV)
    lam = torch.tensor([0.1, 0.27], device=DEV)
    t = (torch.randn(B, H, W, generator=g) * 0.1).to(DEV)
    y = torch.empty(B, H, W, device=DEV)
    loss = torch.full((1,), 123.0, device=DEV)  # overwritten, not accumulated
    go = torch.empty(B, H, W, 16, dtype=torch.bfloat16, device=DEV)
    ws = _ws()
    _lib._check(lib.tv_net_dual_head(_vp(o), B, H, W, _vp(lam), _vp(t), _vp(y), _vp(loss), _vp(go),
                                     _vp(ws), ws.numel(), _stream()))
    ry, rloss, rg = ref.head_loss_grad(_np(o)[..., 0], lam.cpu().numpy().astype(np.float64), _np(t))
    np.testing.assert_allclose(y.cpu().numpy(), ry, rtol=0, atol=1e-6)
    assert abs(loss.item() - rloss) <= 1e-5 * rloss
    _bf16_close(_np(go)[..., 0], rg, atol=1e-9)
    assert not go[..., 1:].float().abs().sum().item()
    # dual feasibility: |p_v| <= lambda row by row, p_v recovered from y by a cumulative sum
    p = -np.cumsum(y.cpu().numpy().astype(np.float64), axis=1)
    assert np.all(np.abs(p) <= lam.cpu().numpy()[:, None, None] + 1e-6)


def test_pack_input_and_cast():
    lib = _lib.load()
    f = torch.rand(B, H, W, generator=torch.Generator().manual_seed(11)).to(DEV)
    lam = torch.tensor([0.05, 0.3], device=DEV)
    x = torch.empty(B, H, W, 16, dtype=torch.bfloat16, device=DEV)
    _lib._check(lib.tv_net_pack_input(_vp(f), B, H, W, _vp(lam), _vp(x), _stream()))
    want = torch.zeros(B, H, W, 16)
    want[..., 0] = f.cpu()
    want[..., 1] = lam.cpu().view(B, 1, 1)
    assert torch.equal(x.cpu(), want.to(torch.bfloat16))
    a = torch.randn(1000, generator=torch.Generator().manual_seed(12)).to(DEV) * 100
    out = torch.empty(1000, dtype=torch.bfloat16, device=DEV)
    _lib._check(lib.tv_net_cast_bf16(_vp(a), 1000, _vp(out), _stream()))
    assert torch.equal(out.cpu(), a.cpu().to(torch.bfloat16))  # round to nearest even


def test_adam_against_reference():
    lib = _lib.load()
    rng = np.random.default_rng(13)
    n = 5000
    w0, m0, v0 = rng.normal(size=n), rng.normal(size=n) * 0.01, rng.uniform(size=n) * 1e-4
    g0 = rng.normal(size=n)
    w, m, v, g = (torch.from_numpy(a.astype(np.float32)).to(DEV) for a in (w0, m0, v0, g0))
    w16 = torch.empty(n, dtype=torch.bfloat16, device=DEV)
    _lib._check(lib.tv_net_adam(_vp(w), _vp(m), _vp(v), _vp(g), n, 1e-3, 0.9, 0.999, 1e-8, 7,
                                _vp(w16), _stream()))
    # the kernel receives the hyperparameters as FP32: give the reference the same values
    lr, b1, b2, eps = (float(np.float32(a)) for a in (1e-3, 0.9, 0.999, 1e-8))
    rw, rm, rv = ref.adam_step(w0.astype(np.float32), m0.astype(np.float32), v0.astype(np.float32),
                               g0.astype(np.float32), lr, b1, b2, eps, 7)
    np.testing.assert_allclose(w.cpu().numpy(), rw, rtol=0, atol=1e-6)
    # FP32 rounding: a few units in the last place of |m| <= 0.3 and of v <= 1e-3
    np.testing.assert_allclose(m.cpu().numpy(), rm, rtol=1e-6, atol=2e-8)
    np.testing.assert_allclose(v.cpu().numpy(), rv, rtol=1e-6, atol=1e-11)
    assert not g.abs().sum().item()  # cleared for the next accumulation
    assert torch.equal(w16, w.to(torch.bfloat16))


def test_train_step_gradient_against_reference():
    """The whole network's gradient (forward in BF16, backward through all four layers and
    the head) against float64 autograd on the same BF16 weights."""
    net = learned.WarmStartNet(DEV, seed=1)
    # a less trivial last layer than the initial one, so every layer gets gradient
    net.params[net.offsets[-1][0]:net.offsets[-1][1]] *= 10.0
    net._refresh_bf16()
    f = torch.stack([torch.from_numpy(synth.warm_start_sample(H, W, s)[0]) for s in (1, 2)]).to(DEV)
    lam = torch.tensor([0.12, 0.21], device=DEV)
    t = (torch.randn(B, H, W, generator=torch.Generator().manual_seed(14)) * 0.05).to(DEV)
    loss = net.loss_and_grad(f, lam, t).item()
    params = []
    w16 = net.params_bf16.float().cpu().numpy().astype(np.float64)
    p32 = net.params.cpu().numpy().astype(np.float64)
    for (cin, cout, _), (w_off, b_off) in zip(learned.LAYERS, net.offsets):
        params.append((w16[w_off:w_off + cout * 9 * cin].reshape(cout, 3, 3, cin),
                       p32[b_off:b_off + cout]))
    args = (params, f.cpu().numpy(), lam.cpu().numpy(), t.cpu().numpy())
    # (1) against the reference that rounds to BF16 where the GPU stores BF16: only the
    # FP32 accumulation order differs (and the rare BF16 rounding it flips)
    eloss, egrads, _ = ref.loss_and_grads_bf16_storage(*args)
    # (2) against plain float64: BF16 storage of activations and backward signals costs a
    # few per cent of the gradient at this small size (about 5 % measured in emulation)
    rloss, rgrads, _ = ref.loss_and_grads(*args)
    assert abs(loss - eloss) <= 1e-4 * eloss and abs(loss - rloss) <= 1e-2 * rloss
    for (gw, gb), (ew, eb), (rw, rb) in zip(net.layer_grads(), egrads, rgrads):
        gw, gb = gw.cpu().numpy(), gb.cpu().numpy()
        for got, emu, want in ((gw, ew, rw), (gb, eb, rb)):
            assert np.linalg.norm(got - emu) <= 5e-3 * np.linalg.norm(emu)
            cos = (got * want).sum() / (np.linalg.norm(got) * np.linalg.norm(want))
            assert cos > 0.995
            assert np.linalg.norm(got - want) <= 0.12 * np.linalg.norm(want)


def test_predict_dual_is_feasible_and_deterministic():
    net = learned.WarmStartNet(DEV, seed=2)
    f = torch.from_numpy(synth.warm_start_sample(64, 96, 5)[0]).to(DEV)
    y1 = net.predict_dual(f, 0.2).clone()
    y2 = net.predict_dual(f, 0.2)
    assert torch.equal(y1, y2) and y1.shape == (1, 64, 96)
    p = -torch.cumsum(y1.double(), dim=1)
    assert p.abs().max().item() <= 0.2 + 1e-6


def test_checkpoint_round_trip():
    net = learned.WarmStartNet(DEV, seed=3)
    f, lam, y = learned.make_dataset([30, 31], H=48, W=64, device=DEV, tol=1e-5, max_iters=200)
    net.train_step(f, lam, y)
    sd = net.state_dict()
    net2 = learned.WarmStartNet(DEV, seed=99)
    net2.load_state_dict(sd)
    assert torch.equal(net2.params, net.params) and torch.equal(net2.params_bf16, net.params_bf16)
    l1 = net.train_step(f, lam, y).item()
    l2 = net2.train_step(f, lam, y).item()
    assert l1 == l2 and torch.equal(net.params, net2.params)


def test_training_reduces_iterations():
    """A short training run on 64 images of 128 x 128 (targets from the plain solver)
    lowers the mean number of outer iterations to gap 1e-4 on 8 held-out images."""
    net = learned.WarmStartNet(DEV, seed=0, lr=2e-3)
    f, lam, y = learned.make_dataset(range(10000, 10064), H=128, W=128, device=DEV)
    hist = learned.train(net, f, lam, y, epochs=25, batch=8)
    assert hist[-1] < 0.5 * hist[0]
    summary, rows = learned.evaluate(net, range(20000, 20008), H=128, W=128, reps=1)
    assert summary["all_converged"]
    assert summary["iters_warm"] < summary["iters_zero"]


def test_poor_network_falls_back_at_the_first_check():
    """A deliberately poor network (random weights set on the host, the output layer
    scaled so that every p_v = lambda * tanh(o) sits near +-lambda with a random sign)
    is judged by the plain method after the first check: the solve returns to y^0 = 0
    there and converges, at the cost of two short runs of first_check iterations, not
    after max_iters."""
    net = learned.WarmStartNet(DEV, seed=11)
    g = torch.Generator().manual_seed(5)
    with torch.no_grad():
        w_last, b_last = net.layer_params()[-1]
        w_last.copy_((torch.randn(w_last.shape, generator=g) * 5.0).to(DEV))
        b_last.zero_()
    net._refresh_bf16()
    f = torch.from_numpy(synth.warm_start_sample(128, 128, 20001)[0]).to(DEV)
    lam = 0.15
    p = -torch.cumsum(net.predict_dual(f, lam)[0].double(), dim=0)
    assert p.abs().mean().item() > 0.5 * lam  # the warm start is far from y = 0
    _, it_zero, _, ok_zero = _lib.tv2d_denoise(f, lam=lam, tol=1e-4, max_iters=200)
    x, it, gap, ok, fb = learned.denoise_warm(net, f, lam, tol=1e-4, max_iters=200,
                                              first_check=3)
    assert ok_zero and ok and fb
    assert it <= 3 + 3 + it_zero
    assert gap <= 1e-4


@pytest.mark.parametrize("grouped", [False, True])
@pytest.mark.parametrize("shape", [(1, 96, 80), (2, 37, 53), (1, 512, 512), (3, 17, 16)])
def test_inference_layers_match_the_general_path(shape, grouped):
    """The inference path (first layer from the image and lambda directly; NHWC or the
    channel-group layout) against the general kernels (packed input, four convolutions,
    head) on the stored network: equal up to the order of FP32 sums, which can move a
    BF16 activation by one ulp (the bound is the one the smoke check holds the network's
    output to against FP64)."""
    net = learned.load_weights(DEV)
    B, H, W = shape
    f = torch.from_numpy(np.stack([synth.warm_start_sample(H, W, 700 + i)[0] for i in range(B)])).to(DEV)
    lam = torch.tensor([0.08 + 0.05 * i for i in range(B)], dtype=torch.float32, device=DEV)
    y_fast = net.predict_dual(f, lam, grouped=grouped).clone()
    y_ref = net.predict_dual_layers(f, lam).clone()
    err = (y_fast - y_ref).abs().max().item()
    assert err <= 1e-2 * lam.max().item(), err
    # feasibility of the fast path's dual: |p_v| <= lambda on every vertical edge
    p = -torch.cumsum(y_fast.double(), dim=1)
    assert (p.abs() <= lam.double().view(B, 1, 1) + 1e-6).all()
