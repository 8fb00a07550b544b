"""FP64 CPU reference of the dual warm-start network (TEST INFRASTRUCTURE ONLY).

The network is not part of the paper (parity of the learned part is unpinned by
the paper); this module fixes what the GPU kernels must compute, with plain
PyTorch CPU float64 operations, and is pinned by tests against facts that do
not reuse it: a delta kernel is a shift, the head is the adjoint of a difference
operator, gradients match finite differences.

Layout as on the GPU: images (B, H, W); activations NHWC; weights [cout][3][3][cin];
3x3 cross-correlation, stride 1, zero padding 1.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def conv3x3(x_nhwc, w, b=None):
    """conv2d in float64: x (B, H, W, Cin), w (Cout, 3, 3, Cin), b (Cout,) -> (B, H, W, Cout)."""
    x = torch.as_tensor(x_nhwc, dtype=torch.float64).permute(0, 3, 1, 2)
    wt = torch.as_tensor(w, dtype=torch.float64).permute(0, 3, 1, 2)
    bb = None if b is None else torch.as_tensor(b, dtype=torch.float64)
    return F.conv2d(x, wt, bb, padding=1).permute(0, 2, 3, 1)


def pack_input(f, lam):
    """Channel 0 the image, channel 1 its lambda, 2..15 zero."""
    f = torch.as_tensor(f, dtype=torch.float64)
    B, H, W = f.shape
    x = torch.zeros(B, H, W, 16, dtype=torch.float64)
    x[..., 0] = f
    x[..., 1] = torch.as_tensor(lam, dtype=torch.float64).view(B, 1, 1)
    return x


def dual_head(o, lam):
    """p_v = lam tanh(o) on rows 0..H-2 (0 on the last row); y = D_v^T p_v with
    y[r] = p[r-1] - p[r] (p[-1] = 0). o: (B, H, W)."""
    o = torch.as_tensor(o, dtype=torch.float64)
    lam = torch.as_tensor(lam, dtype=torch.float64).view(-1, 1, 1)
    p = lam * torch.tanh(o)
    p = torch.cat([p[:, :-1], torch.zeros_like(p[:, -1:])], dim=1)
    up = torch.cat([torch.zeros_like(p[:, :1]), p[:, :-1]], dim=1)
    return up - p


def forward(params, f, lam):
    """Network forward: returns (y, list of pre-activations, list of inputs per layer).
    params: list of (w, b) for the four layers (cin, cout) = (16,32),(32,32),(32,32),(32,16)."""
    x = pack_input(f, lam)
    pres, ins = [], []
    for li, (w, b) in enumerate(params):
        ins.append(x)
        pre = conv3x3(x, w, b)
        pres.append(pre)
        x = torch.relu(pre) if li < len(params) - 1 else pre
    y = dual_head(pres[-1][..., 0], lam)
    return y, pres, ins


def loss_and_grads(params, f, lam, target):
    """Mean squared error of the head output against target, and its gradients
    (float64 autograd) with respect to every weight and bias."""
    ps = [(torch.tensor(np.asarray(w), dtype=torch.float64, requires_grad=True),
           torch.tensor(np.asarray(b), dtype=torch.float64, requires_grad=True)) for w, b in params]
    y, _, _ = forward(ps, f, lam)
    t = torch.as_tensor(target, dtype=torch.float64)
    loss = ((y - t) ** 2).mean()
    loss.backward()
    return float(loss.detach()), [(w.grad.numpy(), b.grad.numpy()) for w, b in ps], y.detach().numpy()


def conv3x3_grads(x_nhwc, w, dy_nhwc):
    """Gradients of sum(conv3x3(x, w, b) * dy) with respect to x, w and b (float64 autograd)."""
    x = torch.tensor(np.asarray(x_nhwc, dtype=np.float64), requires_grad=True)
    wt = torch.tensor(np.asarray(w, dtype=np.float64), requires_grad=True)
    dy = torch.as_tensor(np.asarray(dy_nhwc, dtype=np.float64))
    (conv3x3(x, wt) * dy).sum().backward()
    return x.grad.numpy(), wt.grad.numpy(), dy.sum(dim=(0, 1, 2)).numpy()


def head_loss_grad(o, lam, target):
    """Head output y, loss mean (y - target)^2 and its gradient with respect to o."""
    ot = torch.tensor(np.asarray(o, dtype=np.float64), requires_grad=True)
    y = dual_head(ot, lam)
    loss = ((y - torch.as_tensor(np.asarray(target, dtype=np.float64))) ** 2).mean()
    loss.backward()
    return y.detach().numpy(), float(loss.detach()), ot.grad.numpy()


def adam_step(w, m, v, g, lr, b1, b2, eps, step):
    """One Adam update (Kingma and Ba, Algorithm 1) in float64; returns (w, m, v)."""
    w, m, v, g = (np.asarray(a, dtype=np.float64) for a in (w, m, v, g))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def _bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    return torch.as_tensor(a, dtype=torch.float64).to(torch.bfloat16).to(torch.float64)


def loss_and_grads_bf16_storage(params, f, lam, target):
    """``loss_and_grads`` with every tensor that the GPU network keeps in bfloat16 rounded
    to bfloat16 where it is stored: the packed input, the hidden activations, the head's
    gradient and the hidden backward signals (after the ReLU mask). Arithmetic stays
    float64, so what remains against the GPU is FP32 accumulation order."""
    ps = [(np.asarray(w, dtype=np.float64), np.asarray(b, dtype=np.float64)) for w, b in params]
    x = _bf16(pack_input(f, lam))
    ins, pres = [], []
    for li, (w, b) in enumerate(ps):
        ins.append(x)
        pre = conv3x3(x, w, b)
        pres.append(pre)
        if li < len(ps) - 1:
            x = _bf16(torch.relu(pre))
    o = pres[-1][..., 0].detach().numpy()
    y, loss, g_o = head_loss_grad(o, lam, target)
    dy = torch.zeros(pres[-1].shape, dtype=torch.float64)
    dy[..., 0] = _bf16(g_o)
    grads = [None] * len(ps)
    for li in range(len(ps) - 1, -1, -1):
        dx, dw, db = conv3x3_grads(ins[li].numpy(), ps[li][0], dy.numpy())
        grads[li] = (dw, db)
        if li > 0:
            dy = _bf16(dx * (pres[li - 1].numpy() > 0))
    return loss, grads, y
