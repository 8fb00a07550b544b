"""Learned dual warm start for the 2D primal-dual iteration (eq. pd of Sec. 6.1).

The iteration accepts any initial dual y^0; a closer one needs fewer outer
iterations. ``WarmStartNet`` is a four-layer 3x3 convolutional network (16 -> 32
-> 32 -> 32 -> 16 channels, ReLU between layers; input channel 0 the noisy image,
channel 1 its lambda, the rest zero) whose output channel 0, o, parametrises a
vertical edge field p_v = lambda * tanh(o) and the dual y^0 = D_v^T p_v. Since
|p_v| <= lambda on every vertical edge, y^0 is always a feasible column dual.

Every operation runs in the library's kernels (``tv_net_*``): BF16 tensor-core
convolutions with FP32 accumulation (forward, backward-data, backward-weight),
the head and its gradient, the BF16 cast and Adam; torch only holds the
buffers. Training targets are the duals that the plain solver (zero start, tight
tolerance) returns; the loss is the mean squared error of y^0 against them.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time

import numpy as np
import torch

from . import _lib, synth

# (input channels, output channels, ReLU) of each layer
LAYERS = ((16, 32, True), (32, 32, True), (32, 32, True), (32, 16, False))
_ALIGN = 64  # parameter blocks start on 64-element boundaries (16-byte aligned BF16 views)


def _round_up(n, a=_ALIGN):
    return (n + a - 1) // a * a


def _layout():
    """Offsets (elements) of each layer's weights [cout][3][3][cin] and biases [cout]
    in the flat parameter vector, and its total length."""
    offs, pos = [], 0
    for cin, cout, _ in LAYERS:
        w_off = pos
        pos = _round_up(pos + cout * 9 * cin)
        b_off = pos
        pos = _round_up(pos + cout)
        offs.append((w_off, b_off))
    return offs, pos


def _vp(t, offset_elems=0):
    return ctypes.c_void_p(t.data_ptr() + offset_elems * t.element_size())


class WarmStartNet:
    """The warm-start network with FP32 master parameters, their BF16 copy and Adam state."""

    def __init__(self, device="cuda:0", seed: int = 0, lr: float = 1e-3, betas=(0.9, 0.999),
                 eps: float = 1e-8):
        _lib._require_cuda()
        self.lib = _lib.load()
        self.device = torch.device(device)
        self.lr, self.betas, self.eps = float(lr), tuple(betas), float(eps)
        self.offsets, self.numel = _layout()
        gen = torch.Generator().manual_seed(int(seed))
        flat = torch.zeros(self.numel, dtype=torch.float32)
        for li, ((cin, cout, _), (w_off, _)) in enumerate(zip(LAYERS, self.offsets)):
            fan_in = 9 * (2 if li == 0 else cin)  # layer 0 sees two non-zero channels
            std = math.sqrt(2.0 / fan_in) * (0.1 if li == len(LAYERS) - 1 else 1.0)
            w = torch.randn(cout, 3, 3, cin, generator=gen) * std
            if li == 0:
                w[..., 2:] = 0.0
            flat[w_off:w_off + w.numel()] = w.reshape(-1)
        self.params = flat.to(self.device)
        self.params_bf16 = torch.empty(self.numel, dtype=torch.bfloat16, device=self.device)
        self.grad = torch.zeros(self.numel, dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.grad)
        self.v = torch.zeros_like(self.grad)
        self.step = 0
        self.meta = {}
        # inference activations in the channel-group layout on the TMA-fed tcgen05 kernel
        self.grouped_inference = True
        self._flip = torch.empty(32 * 9 * 32, dtype=torch.bfloat16, device=self.device)
        self._bufs = {}
        self._refresh_bf16()

    # ------------------------------------------------------------------ state --
    def _refresh_bf16(self):
        _lib._check(self.lib.tv_net_cast_bf16(_vp(self.params), self.numel, _vp(self.params_bf16),
                                              _lib._stream(self.device)))

    def state_dict(self):
        return {"params": self.params.detach().cpu().clone(), "m": self.m.cpu().clone(),
                "v": self.v.cpu().clone(), "step": self.step, "lr": self.lr,
                "betas": self.betas, "eps": self.eps, "layers": LAYERS}

    def load_state_dict(self, sd):
        if tuple(map(tuple, sd["layers"])) != LAYERS or sd["params"].numel() != self.numel:
            raise ValueError("checkpoint of a different network")
        self.params.copy_(sd["params"])
        self.m.copy_(sd["m"])
        self.v.copy_(sd["v"])
        self.step = int(sd["step"])
        self.lr, self.betas, self.eps = float(sd["lr"]), tuple(sd["betas"]), float(sd["eps"])
        self.grad.zero_()
        self._refresh_bf16()

    def layer_params(self):
        """The FP32 master weights (cout, 3, 3, cin) and biases (cout,) of each layer (views)."""
        out = []
        for (cin, cout, _), (w_off, b_off) in zip(LAYERS, self.offsets):
            out.append((self.params[w_off:w_off + cout * 9 * cin].view(cout, 3, 3, cin),
                        self.params[b_off:b_off + cout]))
        return out

    def layer_grads(self):
        out = []
        for (cin, cout, _), (w_off, b_off) in zip(LAYERS, self.offsets):
            out.append((self.grad[w_off:w_off + cout * 9 * cin].view(cout, 3, 3, cin),
                        self.grad[b_off:b_off + cout]))
        return out

    # ---------------------------------------------------------------- buffers --
    def _buffers(self, B, H, W, train):
        key = (B, H, W, train)
        bufs = self._bufs.get(key)
        if bufs is None:
            dev, bf = self.device, torch.bfloat16
            n = B * H * W
            nws = self.lib.tv_net_workspace_size(B, H, W)
            if nws == 0:
                raise ValueError(f"unsupported batch shape {(B, H, W)}")
            bufs = {"x0": torch.empty(n * 16, dtype=bf, device=dev),
                    "ws": torch.empty(nws, dtype=torch.uint8, device=dev),
                    "o": torch.empty(n * 16, dtype=torch.float32, device=dev),
                    "y": torch.empty(B, H, W, dtype=torch.float32, device=dev),
                    "loss": torch.zeros(1, dtype=torch.float32, device=dev)}
            bufs["acts"] = [torch.empty(n * cout, dtype=bf, device=dev) for _, cout, _ in LAYERS[:-1]]
            if train:
                bufs["pres"] = [torch.empty(n * cout, dtype=torch.float32, device=dev)
                                for _, cout, _ in LAYERS[:-1]]
                bufs["g_o"] = torch.empty(n * 16, dtype=bf, device=dev)
                bufs["g_a"] = torch.empty(n * 32, dtype=bf, device=dev)
                bufs["g_b"] = torch.empty(n * 32, dtype=bf, device=dev)
            self._bufs = {key: bufs}  # keep one shape at a time
        return bufs

    # ---------------------------------------------------------------- forward --
    def _forward(self, f, lam, bufs, train):
        B, H, W = f.shape
        s = _lib._stream(self.device)
        lib = self.lib
        _lib._check(lib.tv_net_pack_input(_vp(f), B, H, W, _vp(lam), _vp(bufs["x0"]), s))
        x = bufs["x0"]
        for li, ((cin, cout, relu), (w_off, b_off)) in enumerate(zip(LAYERS, self.offsets)):
            last = li == len(LAYERS) - 1
            pre = bufs["o"] if last else (bufs["pres"][li] if train else None)
            act = None if last else bufs["acts"][li]
            _lib._check(lib.tv_net_conv3x3(_vp(x), B, H, W, cin, _vp(self.params_bf16, w_off),
                                           _vp(self.params, b_off), cout, int(relu), _lib._ptr(pre),
                                           _lib._ptr(act), s))
            x = act

    def predict_dual(self, f, lam, grouped=None):
        """Warm start y^0 (B, H, W) for images f (B, H, W) with per-image lambdas
        ``lam`` (a float, a sequence or a (B,) float32 CUDA tensor). The result lives in
        a buffer of the network that the next call overwrites.

        Inference takes the specialised first layer (two non-zero input channels, no
        packed input); the other layers and the head are the general kernels. With
        ``grouped`` (default ``self.grouped_inference``) the activations are kept in the
        channel-group layout, every layer runs on tcgen05 (the first from the image rows,
        the others fed by TMA) and the last layer's epilogue applies the head.
        ``predict_dual_layers`` computes the same through the kernels of training."""
        f, lam = self._inputs(f, lam)
        B, H, W = f.shape
        bufs = self._buffers(B, H, W, train=False)
        s = _lib._stream(self.device)
        lib = self.lib
        grouped = self.grouped_inference if grouped is None else bool(grouped)
        conv = lib.tv_net_conv3x3_grouped if grouped else lib.tv_net_conv3x3
        w0, b0 = self.offsets[0]
        _lib._check(lib.tv_net_first_layer(_vp(f), B, H, W, _vp(lam), _vp(self.params_bf16, w0),
                                           _vp(self.params, b0), _vp(bufs["acts"][0]),
                                           int(grouped), s))
        x = bufs["acts"][0]
        for li in range(1, len(LAYERS)):
            (cin, cout, relu), (w_off, b_off) = LAYERS[li], self.offsets[li]
            last = li == len(LAYERS) - 1
            if last and grouped:  # epilogue keeps channel 0 and applies the head
                _lib._check(lib.tv_net_conv3x3_dual_head(
                    _vp(x), B, H, W, cin, _vp(self.params_bf16, w_off), _vp(self.params, b_off),
                    _vp(lam), _vp(bufs["o"]), _vp(bufs["y"]), s))
                return bufs["y"]
            _lib._check(conv(_vp(x), B, H, W, cin, _vp(self.params_bf16, w_off),
                             _vp(self.params, b_off), cout, int(relu),
                             _vp(bufs["o"]) if last else None,
                             None if last else _vp(bufs["acts"][li]), s))
            x = None if last else bufs["acts"][li]
        _lib._check(lib.tv_net_dual_head(_vp(bufs["o"]), B, H, W, _vp(lam), None, _vp(bufs["y"]),
                                         None, None, None, 0, s))
        return bufs["y"]

    def predict_dual_layers(self, f, lam):
        """predict_dual through the general kernels (packed input, four convolutions,
        the head): the reference the specialised inference path is checked against."""
        f, lam = self._inputs(f, lam)
        B, H, W = f.shape
        bufs = self._buffers(B, H, W, train=False)
        self._forward(f, lam, bufs, train=False)
        _lib._check(self.lib.tv_net_dual_head(_vp(bufs["o"]), B, H, W, _vp(lam), None,
                                              _vp(bufs["y"]), None, None, None, 0,
                                              _lib._stream(self.device)))
        return bufs["y"]

    def _inputs(self, f, lam):
        squeeze = f.dim() == 2
        if squeeze:
            f = f.unsqueeze(0)
        _lib._require_cuda(f)
        B = f.shape[0]
        if not torch.is_tensor(lam):
            lam = torch.tensor(np.broadcast_to(np.asarray(lam, dtype=np.float32), (B,)).copy(),
                               device=self.device)
        _lib._require_cuda(lam)
        if lam.numel() != B:
            raise ValueError("one lambda per image")
        return f.contiguous(), lam.contiguous()

    # ----------------------------------------------------------------- train --
    def loss_and_grad(self, f, lam, target):
        """Forward, loss (device scalar) and backward: the gradient is ADDED to
        ``self.grad`` (cleared by each optimiser step)."""
        f, lam = self._inputs(f, lam)
        target = target.reshape(f.shape)
        _lib._require_cuda(target)
        B, H, W = f.shape
        bufs = self._buffers(B, H, W, train=True)
        s = _lib._stream(self.device)
        lib = self.lib
        self._forward(f, lam, bufs, train=True)
        ws, nws = bufs["ws"], bufs["ws"].numel()
        _lib._check(lib.tv_net_dual_head(_vp(bufs["o"]), B, H, W, _vp(lam), _vp(target),
                                         _vp(bufs["y"]), _vp(bufs["loss"]), _vp(bufs["g_o"]),
                                         _vp(ws), nws, s))
        dy = bufs["g_o"]
        spare = [bufs["g_a"], bufs["g_b"]]
        for li in range(len(LAYERS) - 1, -1, -1):
            cin, cout, _ = LAYERS[li]
            w_off, b_off = self.offsets[li]
            x_in = bufs["x0"] if li == 0 else bufs["acts"][li - 1]
            _lib._check(lib.tv_net_conv3x3_backward_weight(_vp(x_in), _vp(dy), B, H, W, cin, cout,
                                                           _vp(self.grad, w_off),
                                                           _vp(self.grad, b_off), _vp(ws), nws,
                                                           s))
            if li > 0:
                dx = spare[li % 2]
                _lib._check(lib.tv_net_conv3x3_backward_data(_vp(dy), B, H, W, cout,
                                                             _vp(self.params_bf16, w_off), cin,
                                                             _vp(bufs["pres"][li - 1]), _vp(dx),
                                                             _vp(self._flip), s))
                dy = dx
        return bufs["loss"]

    def optimizer_step(self):
        self.step += 1
        _lib._check(self.lib.tv_net_adam(_vp(self.params), _vp(self.m), _vp(self.v),
                                         _vp(self.grad), self.numel, self.lr, self.betas[0],
                                         self.betas[1], self.eps, self.step,
                                         _vp(self.params_bf16), _lib._stream(self.device)))

    def train_step(self, f, lam, target):
        loss = self.loss_and_grad(f, lam, target)
        self.optimizer_step()
        return loss


# --------------------------------------------------------------- data + eval --
def make_dataset(seeds, H=512, W=512, device="cuda:0", tol=1e-6, max_iters=400, chunk=32,
                 lam_range=(0.05, 0.3)):
    """Images of ``synth.warm_start_sample`` and the duals the plain solver (zero
    start) reaches on them at tolerance ``tol``. Returns (f (N,H,W), lam (N,), y* (N,H,W))
    on the device."""
    seeds = list(seeds)
    N = len(seeds)
    dev = torch.device(device)
    f = torch.empty(N, H, W, dtype=torch.float32, device=dev)
    y = torch.empty_like(f)
    lams = np.empty(N, dtype=np.float32)
    for i, sd in enumerate(seeds):
        img, lam = synth.warm_start_sample(H, W, sd, lam_range)
        f[i].copy_(torch.from_numpy(img))
        lams[i] = lam
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        _lib.tv2d_denoise_batched([f[i] for i in range(a, b)], [float(v) for v in lams[a:b]],
                                  max_iters=max_iters, tol=tol,
                                  y_outs=[y[i] for i in range(a, b)])
    return f, torch.from_numpy(lams).to(dev), y


def train(net, f, lam, target, epochs=10, batch=8, seed=0, log=None):
    """Mini-batch Adam on a dataset from ``make_dataset``; returns the mean loss per epoch."""
    N = f.shape[0]
    rng = np.random.default_rng(seed)
    history = []
    for ep in range(epochs):
        order = rng.permutation(N)
        total = torch.zeros((), dtype=torch.float64, device=f.device)
        steps = 0
        for a in range(0, N - batch + 1, batch):
            idx = torch.from_numpy(order[a:a + batch]).to(f.device)
            loss = net.train_step(f.index_select(0, idx), lam.index_select(0, idx),
                                  target.index_select(0, idx))
            total += loss[0]
            steps += 1
        history.append(float(total) / max(steps, 1))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.3e}")
    return history


def denoise_warm(net, f, lam: float, lam_t=None, tol=1e-4, max_iters=400, first_check=6):
    """Solve one (H, W) image from the network's warm start, with the plain method as
    fallback and judge (y^0 = 0 is the method without the network).

    First check, after ``first_check`` outer iterations (the solver's own first batch
    of iterations, after which it reads the device state): a warm-started run that has
    converged is returned. Otherwise its per-pixel gap is compared with the zero-init
    curve at the same iteration, i.e. the gap the plain method reaches from y^0 = 0
    after as many iterations on this image. A non-finite gap, or one above the plain
    method's, sends the solve back to y^0 = 0 right there (the plain run is continued
    to the tolerance); a warm start that is ahead is run to the tolerance. A bad network
    thus costs at most two short runs of ``first_check`` iterations. ``lam_t``: the same
    lambda as a (1,) CUDA tensor (made here if None).

    Returns (x, outer iterations of every run, gap, converged, used_fallback)."""
    if lam_t is None:
        lam_t = torch.tensor([lam], dtype=torch.float32, device=f.device)
    y0 = net.predict_dual(f, lam_t)[0]
    k1 = max(1, min(int(first_check), int(max_iters)))
    x, it, gap, ok = _lib.tv2d_denoise(f, lam=float(lam), y0=y0, tol=tol, max_iters=k1)
    if ok and math.isfinite(gap):
        return x, it, gap, ok, False
    if math.isfinite(gap):
        # the zero-init curve at the first check
        xz, itz, gz, okz = _lib.tv2d_denoise(f, lam=float(lam), tol=tol, max_iters=k1)
        if okz:
            return xz, it + itz, gz, okz, True
        if gap <= gz:
            x, it2, gap, ok = _lib.tv2d_denoise(f, lam=float(lam), y0=y0, tol=tol,
                                                max_iters=max_iters)
            return x, it + itz + it2, gap, ok, False
        it += itz
    x, it2, gap, ok = _lib.tv2d_denoise(f, lam=float(lam), tol=tol, max_iters=max_iters)
    return x, it + it2, gap, ok, True


def evaluate(net, seeds, H=512, W=512, tol=1e-4, max_iters=400, reps=3, device="cuda:0"):
    """Outer iterations and wall time (CUDA events; ms from the call to the result,
    network inference included) to per-pixel gap ``tol``, warm start against zero start,
    per held-out seed."""
    dev = torch.device(device)
    rows = []
    for sd in seeds:
        img, lam = synth.warm_start_sample(H, W, sd)
        f = torch.from_numpy(img).to(dev)
        lam_t = torch.tensor([lam], dtype=torch.float32, device=dev)
        res = {}
        for mode in ("zero", "warm"):
            times = []
            for _ in range(reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                if mode == "zero":
                    _, it, gap, ok = _lib.tv2d_denoise(f, lam=lam, tol=tol, max_iters=max_iters)
                    fb = False
                else:
                    _, it, gap, ok, fb = denoise_warm(net, f, lam, lam_t, tol=tol,
                                                      max_iters=max_iters)
                e1.record()
                torch.cuda.synchronize(dev)
                times.append(e0.elapsed_time(e1))
            res[mode] = (it, float(np.median(times[1:])), gap, ok, fb)
        rows.append({"seed": sd, "lam": lam, "iters_zero": res["zero"][0],
                     "iters_warm": res["warm"][0], "ms_zero": res["zero"][1],
                     "ms_warm": res["warm"][1], "converged": res["zero"][3] and res["warm"][3],
                     "fallback": res["warm"][4]})
    summary = {k: float(np.mean([r[k] for r in rows]))
               for k in ("iters_zero", "iters_warm", "ms_zero", "ms_warm")}
    summary["fallbacks"] = int(sum(r["fallback"] for r in rows))
    summary["all_converged"] = all(r["converged"] for r in rows)
    summary["images"] = len(rows)
    return summary, rows


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warm_start_512.npz")


def save_weights(net, path=WEIGHTS, meta=None):
    """Store the FP32 parameters (and a JSON description of how they were trained)."""
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, params=net.params.cpu().numpy(), layers=np.array(LAYERS),
             meta=json.dumps(meta or {}))


def load_weights(device="cuda:0", path=WEIGHTS):
    """A network with the stored parameters (fresh optimiser state)."""
    data = np.load(path)
    if tuple(map(tuple, data["layers"].tolist())) != LAYERS:
        raise ValueError("weights of a different network")
    net = WarmStartNet(device)
    net.params.copy_(torch.from_numpy(data["params"]))
    net._refresh_bf16()
    net.meta = json.loads(str(data["meta"]))
    return net


def run_experiment(n_train=2000, n_eval=200, H=512, W=512, epochs=20, batch=8, lr=2e-3,
                   device="cuda:0", seed=0, save=None, log=print):
    """Train on ``n_train`` images (seeds 10000...) with targets from the plain solver at
    tolerance 1e-6, evaluate on ``n_eval`` held-out seeds (20000...) against the zero
    start. Returns (net, summary)."""
    t0 = time.time()
    f, lam, y = make_dataset(range(10000, 10000 + n_train), H=H, W=W, device=device)
    torch.cuda.synchronize(device)
    t_data = time.time() - t0
    net = WarmStartNet(device, seed=seed, lr=lr)
    t0 = time.time()
    hist = train(net, f, lam, y, epochs=epochs, batch=batch, seed=seed, log=log)
    torch.cuda.synchronize(device)
    t_train = time.time() - t0
    del f, lam, y
    summary, _ = evaluate(net, range(20000, 20000 + n_eval), H=H, W=W, device=device)
    summary.update({"train_images": n_train, "epochs": epochs, "batch": batch, "lr": lr,
                    "size": [H, W], "final_loss": hist[-1], "first_loss": hist[0],
                    "data_s": round(t_data, 1), "train_s": round(t_train, 1),
                    "steps": net.step})
    if save:
        save_weights(net, save, summary)
    return net, summary


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser(description="train and evaluate the dual warm-start network")
    ap.add_argument("--train", type=int, default=2000)
    ap.add_argument("--eval", type=int, default=200)
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--save", default=None, help="where to store the trained weights (.npz)")
    a = ap.parse_args()
    _, s = run_experiment(a.train, a.eval, a.size, a.size, a.epochs, a.batch, a.lr, save=a.save)
    print(json.dumps(s))
