"""ctypes binding of ``libtv.so`` (the C ABI declared in ``include/tv.h``).

Argument marshalling only: every step of every solve runs in the library's
CUDA kernels. Tensors are torch CUDA tensors; their device pointers and the
current torch stream are handed to the C entry points. Workspaces are
allocated here with torch and reused across calls of the same size.

There is no CPU fallback: if the library cannot be built or loaded, or no CUDA
device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

(TV_OK, TV_ERR_INVALID, TV_ERR_CUDA, TV_ERR_NOT_CONVERGED, TV_ERR_TIMEOUT, TV_ERR_NOMEM,
 TV_ERR_CAPACITY) = range(7)

_lock = threading.Lock()
_lib = None

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_sz = ctypes.c_size_t

class ImageDesc(ctypes.Structure):
    """tv_image_desc of include/tv.h: one image of a batch (device pointers)."""
    _fields_ = [("img", ctypes.c_void_p), ("H", ctypes.c_int64), ("W", ctypes.c_int64),
                ("wh", ctypes.c_void_p), ("wv", ctypes.c_void_p), ("lam", ctypes.c_float),
                ("y0", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y_out", ctypes.c_void_p)]


# name -> (restype, argtypes), mirroring include/tv.h
SIGNATURES = {
    "tv_last_error": (ctypes.c_char_p, []),
    "tv_version": (ctypes.c_int, []),
    "tv_launch_count": (_i64, []),
    "tv_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "tv_profile_read": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(_i64)]),
    "tv_chain_workspace_size": (_sz, [_i64, _i64]),
    "tv_chain_solve": (ctypes.c_int, [_p, _p, ctypes.c_float, _p, _i64, _i64, _p, _p, _sz, _p]),
    "tv_chain_solve_noalloc": (ctypes.c_int, [_p, _p, ctypes.c_float, _p, _i64, _i64, _p, _p]),
    "tv_chain_solve_backward": (ctypes.c_int, [_p, _p, _p, _i64, _i64, _p, _p, _p, _sz, _p]),
    "tv_columns_workspace_size": (_sz, [_i64, _i64]),
    "tv_chain_solve_columns": (ctypes.c_int,
                               [_p, _p, ctypes.c_float, _i64, _i64, _i64, _p, _p, _sz, _p]),
    "tv_workspace_status": (ctypes.c_int, [_p, _p, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(_i64)]),
    "tv2d_workspace_size": (_sz, [_i64, _i64, ctypes.c_int]),
    "tv2d_batched_workspace_size": (_sz, [ctypes.POINTER(ImageDesc), ctypes.c_int, ctypes.c_int]),
    "tv2d_denoise_batched": (ctypes.c_int, [ctypes.POINTER(ImageDesc), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_double), _p, _sz, _p]),
    "tv_set_batched_warps": (ctypes.c_int, [ctypes.c_int]),
    "tv2d_batched_last_mode": (ctypes.c_int, []),
    "tv_set_batched_graph": (ctypes.c_int, [ctypes.c_int]),
    "tv_set_coop_max_chains": (ctypes.c_int, [_i64]),
    "tv_chain_pq_workspace_size": (_sz, [_i64, _i64]),
    "tv_chain_nonconvex_workspace_size": (_sz, [_i64, _i64, _i64, ctypes.c_int]),
    "tv_chain_solve_nonconvex": (ctypes.c_int, [_p, _p, _p, ctypes.c_int, _p, _p, ctypes.c_float,
                                                ctypes.c_float, _p, ctypes.c_float, _p,
                                                ctypes.c_float, _p, _i64, _i64, _i64,
                                                ctypes.c_int, _p, _p, _p, _sz, _p]),
    "tv_chain_solve_pq": (ctypes.c_int, [_p, _p, _p, ctypes.c_float, _p, _p, ctypes.c_float, _p,
                                         _i64, _i64, _p, _p, _sz, _p]),
    "tv2d_lagrangian_workspace_size": (_sz, [_i64, _i64]),
    "tv2d_denoise_lagrangian": (ctypes.c_int, [_p, _i64, _i64, _p, _p, ctypes.c_float,
                                               ctypes.c_float, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_int, _p, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_double), _p, _sz, _p]),
    "tv2d_l1_workspace_size": (_sz, [_i64, _i64]),
    "tv2d_denoise_l1": (ctypes.c_int, [_p, _i64, _i64, _p, _p, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_int, _p,
                                       ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double), _p, _sz, _p]),
    "tv_chain_solve_general": (ctypes.c_int, [_p, _p, _p, _p, _p, _i64, _i64, _p, _p, _sz, _p]),
    "tv_set_coop_split": (ctypes.c_int, [ctypes.c_int]),
    "tv_set_thread_split": (ctypes.c_int, [ctypes.c_int]),
    "tv_set_programmatic_launch": (ctypes.c_int, [ctypes.c_int]),
    "tv_net_set_tensor_path": (ctypes.c_int, [ctypes.c_int]),
    "tv_net_tensor_timeouts": (_i64, []),
    "tv_net_conv3x3": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _p, _p, ctypes.c_int, ctypes.c_int, _p, _p, _p]),
    "tv_net_conv3x3_backward_data": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int, _p, ctypes.c_int, _p, _p, _p,
                                                    _p]),
    "tv_net_workspace_size": (_sz, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "tv_net_conv3x3_backward_weight": (ctypes.c_int, [_p, _p, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      _p, _p, _p, _sz, _p]),
    "tv_net_pack_input": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _p, _p,
                                         _p]),
    "tv_net_dual_head": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _p, _p, _p,
                                        _p, _p, _p, _sz, _p]),
    "tv_net_first_layer": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _p, _p,
                                          _p, _p, ctypes.c_int, _p]),
    "tv_net_conv3x3_dual_head": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, _p, _p, _p, _p, _p, _p]),
    "tv_net_conv3x3_grouped": (ctypes.c_int, [_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, _p, _p, ctypes.c_int, ctypes.c_int,
                                              _p, _p, _p]),
    "tv_net_cast_bf16": (ctypes.c_int, [_p, _i64, _p, _p]),
    "tv_net_adam": (ctypes.c_int, [_p, _p, _p, _p, _i64, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, ctypes.c_int, _p, _p]),
    "tv2d_denoise": (ctypes.c_int, [_p, _i64, _i64, _p, _p, ctypes.c_float, _p, ctypes.c_int,
                                    ctypes.c_double, _p, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double), _p, _sz, _p]),
}


class TVError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tv status {status}: {msg}")
        self.status = status


def load(build_if_needed: bool = True):
    """Load ``libtv.so`` (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_needed and (not os.path.exists(path) or _build.stale()):
                _build.build()
            if not os.path.exists(path):
                raise ImportError(f"libtv.so is not built ({path})")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status):
    if status != TV_OK:
        raise TVError(status, load().tv_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _require_cuda(*tensors):
    if not torch.cuda.is_available():
        raise RuntimeError("the TV library needs a CUDA device; there is no CPU fallback")
    for t in tensors:
        if t is None:
            continue
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("inputs must be contiguous float32 CUDA tensors")


_ws_cache: dict = {}


def workspace(nbytes: int, device, key: str = "default") -> torch.Tensor:
    """A cached uint8 device buffer of at least ``nbytes`` bytes."""
    dev = torch.device(device)
    k = (key, dev.index)
    buf = _ws_cache.get(k)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
        _ws_cache[k] = buf
    return buf


def chain_prox(y, w=None, lam: float = 0.0, offsets=None, max_len: int | None = None,
               out=None, ws=None):
    """Solve eq. 1D-ROF on a batch of contiguous chains.

    ``y``: (B, n) tensor of B chains of length n, or a flat tensor with int64
    ``offsets`` (B+1, on the same device) and ``max_len``. ``w``: per-node edge
    weights laid out like ``y`` (last node of each chain unused), or None for
    the uniform weight ``lam``.
    """
    lib = load()
    _require_cuda(y, w)
    if offsets is None:
        if y.dim() != 2:
            raise ValueError("y must be (num_chains, n) without offsets")
        num_chains, n = y.shape
        max_len = n
        offp = None
    else:
        if offsets.dtype != torch.int64 or not offsets.is_cuda:
            raise ValueError("offsets must be an int64 CUDA tensor")
        num_chains = offsets.numel() - 1
        if max_len is None:
            raise ValueError("max_len is required with offsets")
        offp = _ptr(offsets)
    x = torch.empty_like(y) if out is None else out
    nbytes = lib.tv_chain_workspace_size(num_chains, max_len)
    wsb = ws if ws is not None else workspace(nbytes, y.device, "chain")
    _check(lib.tv_chain_solve(_ptr(y), _ptr(w), float(lam), offp, num_chains, max_len, _ptr(x),
                              _ptr(wsb), wsb.numel(), _stream(y.device)))
    return x


def chain_prox_general(b, wlo, whi, a=None, offsets=None, max_len: int | None = None, out=None,
                       ws=None):
    """General convex chains: argmin sum (a_i x_i^2/2 - b_i x_i) + sum f_i(x_{i+1} - x_i) with
    f_i(d) = wlo_i d (d < 0), whi_i d (d >= 0). ``b``, ``wlo``, ``whi`` (and ``a``, default 1)
    are (num_chains, n) or flat with CSR ``offsets`` (int64 CUDA tensor) and ``max_len``."""
    lib = load()
    _require_cuda(b, wlo, whi, a)
    if offsets is None:
        if b.dim() != 2:
            raise ValueError("b must be (num_chains, n) when offsets is None")
        num_chains, n = b.shape
        max_len = n
    else:
        if max_len is None:
            raise ValueError("max_len is required with offsets")
        num_chains = offsets.numel() - 1
    x = torch.empty_like(b) if out is None else out
    nbytes = lib.tv_chain_workspace_size(num_chains, max_len)
    wsb = ws if ws is not None else workspace(nbytes, b.device, "chain")
    _check(lib.tv_chain_solve_general(_ptr(a), _ptr(b), _ptr(wlo), _ptr(whi), _ptr(offsets),
                                      num_chains, max_len, _ptr(x), _ptr(wsb), wsb.numel(),
                                      _stream(b.device)))
    return x


def chain_prox_pq(b, f, a=None, alpha=1.0, w=None, lam: float = 0.0, offsets=None,
                  max_len: int | None = None, out=None, ws=None):
    """Chains with piecewise-quadratic unaries: argmin sum (a_i x_i^2/2 - b_i x_i +
    alpha_i |x_i - f_i|) + sum w_i |x_{i+1} - x_i|. ``alpha`` and ``w`` are tensors or
    scalars (``lam`` when ``w`` is None); layouts as :func:`chain_prox_general`."""
    lib = load()
    alpha_t = alpha if torch.is_tensor(alpha) else None
    _require_cuda(b, f, a, alpha_t, w)
    if offsets is None:
        if b.dim() != 2:
            raise ValueError("b must be (num_chains, n) when offsets is None")
        num_chains, n = b.shape
        max_len = n
    else:
        if max_len is None:
            raise ValueError("max_len is required with offsets")
        num_chains = offsets.numel() - 1
    x = torch.empty_like(b) if out is None else out
    nbytes = lib.tv_chain_pq_workspace_size(num_chains, max_len)
    wsb = ws if ws is not None else workspace(nbytes, b.device, "pq")
    _check(lib.tv_chain_solve_pq(_ptr(a), _ptr(b), _ptr(alpha_t),
                                 0.0 if alpha_t is not None else float(alpha), _ptr(f), _ptr(w),
                                 float(lam), _ptr(offsets), num_chains, max_len, _ptr(x),
                                 _ptr(wsb), wsb.numel(), _stream(b.device)))
    return x


def chain_prox_nonconvex(uval, uoff=None, ulam=None, sl=-1.0, sr=1.0, w=0.0, C=float("inf"),
                         offsets=None, max_len: int | None = None, max_breakpoints: int = 512,
                         out=None, energy=None, ws=None):
    """Non-convex chains (Sec. 3): argmin sum_i f_i(x_i) + sum_i min(w_i |x_{i+1} - x_i|, C_i)
    with continuous piecewise-linear unaries f_i.

    Unaries: a cost volume ``uval`` of shape (num_chains, n, L) or (num_nodes, L) with
    breakpoints 0..L-1 (``uoff`` None), or CSR ``uoff`` (num_nodes + 1, int64), ``ulam``,
    ``uval`` (flat). ``sl``/``sr`` (end slopes), ``w`` and ``C`` are per-node tensors or
    scalars. Chains: ``offsets`` (CSR over nodes, with ``max_len``) or, without offsets,
    the (num_chains, n) layout of a grid ``uval`` (CSR: one chain). Returns
    ``(x, energy)``: x per node, the optimum energy per chain (float64)."""
    lib = load()
    _require_cuda(*[v for v in (uval, ulam, sl, sr, w, C) if torch.is_tensor(v)])
    for v in (uoff, offsets):
        if v is not None and (not v.is_cuda or v.dtype != torch.int64 or not v.is_contiguous()):
            raise ValueError("uoff and offsets must be contiguous int64 CUDA tensors")
    dev = uval.device
    if uoff is None:
        L = uval.shape[-1]
        num_nodes = uval.numel() // L
        if offsets is None:
            if uval.dim() != 3:
                raise ValueError("uval must be (num_chains, n, L) when offsets is None")
            num_chains, max_len = uval.shape[0], uval.shape[1]
    else:
        L = 0
        num_nodes = uoff.numel() - 1
        if offsets is None:
            num_chains, max_len = 1, num_nodes
    if offsets is not None:
        if max_len is None:
            raise ValueError("max_len is required with offsets")
        num_chains = offsets.numel() - 1
    x = torch.empty(num_nodes, dtype=torch.float32, device=dev) if out is None else out
    e = torch.empty(num_chains, dtype=torch.float64, device=dev) if energy is None else energy
    nbytes = lib.tv_chain_nonconvex_workspace_size(num_nodes, num_chains, max_len,
                                                   int(max_breakpoints))
    wsb = ws if ws is not None else workspace(nbytes, dev, "nonconvex")
    tens = lambda v: v if torch.is_tensor(v) else None
    scal = lambda v: 0.0 if torch.is_tensor(v) else float(v)
    _check(lib.tv_chain_solve_nonconvex(_ptr(uoff), _ptr(ulam), _ptr(uval), int(L),
                                        _ptr(tens(sl)), _ptr(tens(sr)), scal(sl), scal(sr),
                                        _ptr(tens(w)), scal(w), _ptr(tens(C)), scal(C),
                                        _ptr(offsets), num_nodes, num_chains, max_len,
                                        int(max_breakpoints), _ptr(x), _ptr(e), _ptr(wsb),
                                        wsb.numel(), _stream(dev)))
    return x, e


def chain_prox_columns(y, w=None, lam: float = 0.0, out=None, ws=None):
    """Solve eq. 1D-ROF on the columns of a row-major (H, W) tensor."""
    lib = load()
    _require_cuda(y, w)
    H, W = y.shape
    x = torch.empty_like(y) if out is None else out
    nbytes = lib.tv_columns_workspace_size(H, W)
    wsb = ws if ws is not None else workspace(nbytes, y.device, "cols")
    _check(lib.tv_chain_solve_columns(_ptr(y), _ptr(w), float(lam), H, W, W, _ptr(x), _ptr(wsb),
                                      wsb.numel(), _stream(y.device)))
    return x


def chain_prox_backward(x, grad_x, offsets=None, max_len=None, with_w=False, ws=None):
    """Backward of ``chain_prox``: (grad_y, grad_w or None) for upstream ``grad_x``.

    Layouts as in ``chain_prox``; ``grad_w`` has the layout of ``x`` (the entry at a
    chain's last node is zero)."""
    lib = load()
    _require_cuda(x, grad_x)
    if offsets is None:
        num_chains, max_len = x.shape
        offp = None
    else:
        num_chains = offsets.numel() - 1
        if max_len is None:
            raise ValueError("max_len is required with offsets")
        offp = _ptr(offsets)
    gy = torch.empty_like(x)
    gw = torch.zeros_like(x) if with_w else None
    wsb = ws if ws is not None else workspace(256, x.device, "grad")
    _check(lib.tv_chain_solve_backward(_ptr(x), _ptr(grad_x), offp, num_chains, max_len,
                                       _ptr(gy), _ptr(gw), _ptr(wsb), wsb.numel(),
                                       _stream(x.device)))
    return gy, gw


class ChainProxFn(torch.autograd.Function):
    """Differentiable chain TV prox: x = argmin 1/2||x - y||^2 + sum w_e |x_{e+1} - x_e|
    on each row of ``y`` (B, n). ``w`` is a (B, n) tensor of per-node edge weights or a
    Python float; gradients flow to ``y`` and to a tensor ``w``."""

    @staticmethod
    def forward(ctx, y, w):
        if isinstance(w, torch.Tensor):
            x = chain_prox(y.contiguous(), w.contiguous())
        else:
            x = chain_prox(y.contiguous(), lam=float(w))
        ctx.w_is_tensor = isinstance(w, torch.Tensor)
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        need_w = ctx.w_is_tensor and ctx.needs_input_grad[1]
        gy, gw = chain_prox_backward(x, grad_x.contiguous(), with_w=need_w)
        return gy, (gw if need_w else None)


def chain_prox_diff(y, w):
    """Autograd entry point of the chain prox (see ``ChainProxFn``)."""
    return ChainProxFn.apply(y, w)


def workspace_status(ws, device=None):
    """(status, overflowed chains) of a chain workspace; clears the device word."""
    lib = load()
    st = ctypes.c_int(0)
    ov = ctypes.c_int64(0)
    _check(lib.tv_workspace_status(_ptr(ws), _stream(ws.device), ctypes.byref(st),
                                   ctypes.byref(ov)))
    return st.value, ov.value


PROFILE_KINDS = {"chain": 0, "col": 1, "row": 2, "init": 3, "grad": 4}


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().tv_launch_count())


def profile_enable(on: bool = True):
    _check(load().tv_profile_enable(1 if on else 0))


def profile_read(kind: str):
    """(total ms, launches) of one kernel kind since the last read (CUDA events)."""
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().tv_profile_read(PROFILE_KINDS[kind], ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def tv2d_denoise(img, lam: float = 0.1, w_h=None, w_v=None, y0=None, max_iters: int = 200,
                 tol: float = 1e-4, out=None, ws=None):
    """2D TV-l2 (ROF) denoising by the primal-dual Lagrangian decomposition.

    Returns ``(x, iterations, per-pixel gap, converged)``.
    """
    lib = load()
    _require_cuda(img, w_h, w_v, y0)
    H, W = img.shape
    x = torch.empty_like(img) if out is None else out
    nbytes = lib.tv2d_workspace_size(H, W, int(max_iters))
    wsb = ws if ws is not None else workspace(nbytes, img.device, "tv2d")
    it = ctypes.c_int(0)
    gap = ctypes.c_double(0.0)
    st = lib.tv2d_denoise(_ptr(img), H, W, _ptr(w_h), _ptr(w_v), float(lam), _ptr(y0),
                          int(max_iters), float(tol), _ptr(x), ctypes.byref(it),
                          ctypes.byref(gap), _ptr(wsb), wsb.numel(), _stream(img.device))
    if st not in (TV_OK, TV_ERR_NOT_CONVERGED):
        _check(st)
    return x, it.value, gap.value, st == TV_OK


def tv2d_denoise_lagrangian(img, lam: float = 0.1, w_h=None, w_v=None, tau0: float = 10.0,
                            max_iters: int = 500, tol: float = 1e-4, check_every: int = 5,
                            out=None, ws=None):
    """ROF by the symmetric Lagrangian split (x_h, x_v, y) of Sec. 6 with tau_k = tau0 / k.

    Returns ``(x, iterations, per-pixel gap, converged)``.
    """
    lib = load()
    _require_cuda(img, w_h, w_v)
    H, W = img.shape
    x = torch.empty_like(img) if out is None else out
    nbytes = lib.tv2d_lagrangian_workspace_size(H, W)
    wsb = ws if ws is not None else workspace(nbytes, img.device, "lagrangian")
    it = ctypes.c_int(0)
    gap = ctypes.c_double(0.0)
    st = lib.tv2d_denoise_lagrangian(_ptr(img), H, W, _ptr(w_h), _ptr(w_v), float(lam),
                                     float(tau0), int(max_iters), float(tol), int(check_every),
                                     _ptr(x), ctypes.byref(it), ctypes.byref(gap), _ptr(wsb),
                                     wsb.numel(), _stream(img.device))
    if st not in (TV_OK, TV_ERR_NOT_CONVERGED):
        _check(st)
    return x, it.value, gap.value, st == TV_OK


def tv2d_denoise_l1(img, lam: float = 0.55, w_h=None, w_v=None, tau: float = 0.1,
                    max_iters: int = 300, tol: float = 0.0, check_every: int = 10, out=None,
                    ws=None):
    """TV-l1 denoising min TV(x) + ||x - f||_1 (Sec. 6) by eq. pd at constant steps tau,
    1/tau: column chains for the dual, piecewise-quadratic row chains for the primal.

    Returns ``(x, iterations, energy, converged)``; with ``tol = 0`` exactly
    ``max_iters`` iterations run and ``converged`` is True.
    """
    lib = load()
    _require_cuda(img, w_h, w_v)
    H, W = img.shape
    x = torch.empty_like(img) if out is None else out
    nbytes = lib.tv2d_l1_workspace_size(H, W)
    wsb = ws if ws is not None else workspace(nbytes, img.device, "l1")
    it = ctypes.c_int(0)
    en = ctypes.c_double(0.0)
    st = lib.tv2d_denoise_l1(_ptr(img), H, W, _ptr(w_h), _ptr(w_v), float(lam), float(tau),
                             int(max_iters), float(tol), int(check_every), _ptr(x),
                             ctypes.byref(it), ctypes.byref(en), _ptr(wsb), wsb.numel(),
                             _stream(img.device))
    if st not in (TV_OK, TV_ERR_NOT_CONVERGED):
        _check(st)
    return x, it.value, en.value, st == TV_OK


def tv2d_denoise_batched(images, lams, w_hs=None, w_vs=None, y0s=None, max_iters: int = 200,
                         tol: float = 1e-4, outs=None, ws=None, y_outs=None):
    """Denoise a list of (H_i, W_i) images of any sizes in one batched solve.

    ``lams``: per-image uniform weights (used where the image has no w_h / w_v);
    ``w_hs`` / ``w_vs`` / ``y0s``: optional per-image lists (entries may be None).
    Returns ``(xs, iterations, per-pixel gaps, all converged)``.
    """
    lib = load()
    n = len(images)
    w_hs = w_hs or [None] * n
    w_vs = w_vs or [None] * n
    y0s = y0s or [None] * n
    y_outs = y_outs or [None] * n
    _require_cuda(*images, *[t for t in w_hs + w_vs + y0s if t is not None])
    xs = outs if outs is not None else [torch.empty_like(im) for im in images]
    descs = (ImageDesc * n)()
    for m, im in enumerate(images):
        H, W = im.shape
        descs[m] = ImageDesc(im.data_ptr(), H, W,
                             w_hs[m].data_ptr() if w_hs[m] is not None else None,
                             w_vs[m].data_ptr() if w_vs[m] is not None else None,
                             float(lams[m]),
                             y0s[m].data_ptr() if y0s[m] is not None else None,
                             xs[m].data_ptr(),
                             y_outs[m].data_ptr() if y_outs[m] is not None else None)
    nbytes = lib.tv2d_batched_workspace_size(descs, n, int(max_iters))
    if nbytes == 0:
        raise ValueError("malformed image batch")
    wsb = ws if ws is not None else workspace(nbytes, images[0].device, "batched")
    iters = (ctypes.c_int * n)()
    gaps = (ctypes.c_double * n)()
    st = lib.tv2d_denoise_batched(descs, n, int(max_iters), float(tol), iters, gaps, _ptr(wsb),
                                  wsb.numel(), _stream(images[0].device))
    if st not in (TV_OK, TV_ERR_NOT_CONVERGED):
        _check(st)
    return xs, list(iters), list(gaps), st == TV_OK


def set_batched_warps(wpb: int):
    _check(load().tv_set_batched_warps(int(wpb)))


def set_batched_graph(on: bool):
    _check(load().tv_set_batched_graph(int(bool(on))))


def set_coop_split(mode: int):
    """0: one warp per chain from one end; 1: two 16-lane halves from the middle (default);
    2: two warps from the middle."""
    _check(load().tv_set_coop_split(int(mode)))


def set_thread_split(mode: int):
    """Kernel of the one-thread-per-chain path of ``chain_prox`` for chains of 64 nodes or
    more: 2 (the default) middle-rooted chains, a thread per half, each lane updating its
    message at its own pace with a fixed-shape step; 1 the same halves with the lanes'
    updates in step; 0 one thread per chain from one end."""
    _check(load().tv_set_thread_split(int(mode)))


def set_programmatic_launch(on: bool):
    """Launch the 2D solvers' kernels (ROF, Lagrangian split, TV-l1) with a programmatic
    dependency on their predecessor (the default) or in plain stream order; results are
    identical."""
    _check(load().tv_set_programmatic_launch(int(bool(on))))


def set_net_tensor_path(mode: int):
    """Forward convolutions of the warm-start network (NHWC) on mma.sync (0), on tcgen05
    with TMEM accumulators (1), or on tcgen05 fed by TMA with warp roles over row strips
    (2). Inference in the channel-group layout always takes the kernel of mode 2."""
    _check(load().tv_net_set_tensor_path(int(mode)))


def set_coop_max_chains(n: int):
    _check(load().tv_set_coop_max_chains(int(n)))
