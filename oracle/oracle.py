"""ctypes wrapper of the plain FP64 C oracle (``tv_oracle.c``).

TEST INFRASTRUCTURE ONLY. Inputs arrive as float32 or float64 numpy arrays and
are promoted to float64; results come back as float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ``tv_oracle.c`` into ``liboracle.so`` next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.tvo_chain_solve.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _D, _D, _D,
                                            _I64]
            lib.tvo_chain_solve_batch.argtypes = [_D, _D, ctypes.c_double, _I64, ctypes.c_int64,
                                                  _D, ctypes.c_int, _I64]
            lib.tvo_chain_solve_general_batch.argtypes = [_D, _D, _D, _D, _I64, ctypes.c_int64, _D]
            lib.tvo_tv2d_lagrangian.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                 ctypes.c_double, ctypes.c_int, ctypes.c_int, _D,
                                                 ctypes.POINTER(ctypes.c_int), _D]
            lib.tvo_chain_solve_pq_batch.argtypes = [_D, _D, _D, _D, _D, _I64, ctypes.c_int64, _D]
            lib.tvo_tv2d_l1.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ctypes.c_int, _D, _D]
            lib.tvo_chain_solve_nonconvex_batch.argtypes = [_I64, _D, _D, _D, _D, _D, _D, _I64,
                                                            ctypes.c_int64, _D, _D]
            lib.tvo_chain_vjp.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_double, _D, _D]
            lib.tvo_rof_primal.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D,
                                           ctypes.c_double, _D]
            lib.tvo_rof_primal.restype = ctypes.c_double
            lib.tvo_tv2d_pd.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                        _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int), _D, _D]
            _lib = lib
    return _lib


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def chain_solve(c, w=None, lam=0.0, return_records=False):
    """Exact solution of eq. 1D-ROF on one chain: argmin 1/2||x-c||^2 + sum w_e|x_{e+1}-x_e|.

    ``w`` has ``len(c) - 1`` edge weights, or is None for the uniform weight ``lam``.
    With ``return_records`` also returns (lambda^-, lambda^+, largest message length).
    """
    lib = _load()
    c = _f64(c)
    n = c.shape[0]
    w = _f64(w)
    if w is not None and w.shape[0] < max(n - 1, 0):
        raise ValueError("w needs n-1 entries")
    x = np.empty(n)
    lo = np.empty(n) if return_records else None
    hi = np.empty(n) if return_records else None
    m = ctypes.c_int64(0)
    st = lib.tvo_chain_solve(n, _p(c), _p(w), float(lam), _p(x), _p(lo), _p(hi), ctypes.byref(m))
    if st != 0:
        raise RuntimeError(f"oracle chain solve failed: {st}")
    if return_records:
        return x, lo, hi, int(m.value)
    return x


def chain_solve_batch(c, offsets, w=None, lam=0.0, nthreads=None, return_max_len=False):
    """Every chain ``c[offsets[k]:offsets[k+1]]`` solved independently (threaded).

    ``w`` is indexed per node like ``c``; the entry at a chain's last node is unused.
    """
    lib = _load()
    c = _f64(c)
    w = _f64(w)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    nthreads = nthreads or os.cpu_count() or 1
    x = np.empty_like(c)
    m = ctypes.c_int64(0)
    st = lib.tvo_chain_solve_batch(_p(c), _p(w), float(lam), offsets.ctypes.data_as(_I64),
                                   offsets.shape[0] - 1, _p(x), int(nthreads), ctypes.byref(m))
    if st != 0:
        raise RuntimeError(f"oracle batch solve failed: {st}")
    return (x, int(m.value)) if return_max_len else x


def chain_solve_general(a, b, wlo, whi, offsets=None):
    """General convex chains of Sec. 4 / 4.1 (Algorithm 2): unaries a_i x^2/2 - b_i x
    (a_i > 0), pairwise w^-_i d (d < 0) / w^+_i d (d >= 0) on d = x_{i+1} - x_i. Arrays
    of one entry per node (wlo/whi at a chain's last node unused); ``offsets`` CSR
    (default: one chain)."""
    a, b, wlo, whi = (_f64(v) for v in (a, b, wlo, whi))
    n = b.size
    if offsets is None:
        offsets = np.array([0, n], dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    x = np.empty(n, dtype=np.float64)
    st = _load().tvo_chain_solve_general_batch(_p(a), _p(b), _p(wlo), _p(whi),
                                               offsets.ctypes.data_as(_I64), offsets.size - 1,
                                               _p(x))
    if st != 0:
        raise ValueError(f"oracle general chain solve failed ({st})")
    return x


def chain_vjp(x, g, fuse_tol=1e-9, with_w=False):
    """dL/dc (and dL/dw if ``with_w``) of the chain prox at solution ``x`` for
    upstream gradient ``g``; segments are runs with |x_{e+1}-x_e| <= fuse_tol."""
    lib = _load()
    x = _f64(x)
    g = _f64(g)
    n = x.shape[0]
    gc = np.empty(n)
    gw = np.empty(max(n - 1, 0)) if with_w else None
    st = lib.tvo_chain_vjp(n, _p(x), _p(g), float(fuse_tol), _p(gc), _p(gw))
    if st != 0:
        raise RuntimeError("oracle vjp failed")
    return (gc, gw) if with_w else gc


def rof_primal(f, x, w_h=None, w_v=None, lam=0.0):
    """P(x) = 1/2||x-f||^2 + TV_h(x) + TV_v(x) (Sec. 6.1) in float64."""
    lib = _load()
    f = _f64(f)
    x = _f64(x)
    H, W = f.shape
    return lib.tvo_rof_primal(H, W, _p(f), _p(_f64(w_h)), _p(_f64(w_v)), float(lam), _p(x))


def tv2d_pd(f, lam=0.0, w_h=None, w_v=None, y0=None, max_iters=1000, tol=1e-4, tau0=1.0,
            nthreads=None, return_y=False):
    """Accelerated primal-dual ROF solver of eq. pd with row/column chain proxes.

    Returns ``(x, iters, gap_trace, converged)`` (plus the final dual ``y`` if
    ``return_y``); ``gap_trace[k]`` is the per-pixel gap G_k / (H W).
    """
    lib = _load()
    f = _f64(f)
    H, W = f.shape
    nthreads = nthreads or os.cpu_count() or 1
    x = np.empty((H, W))
    y = np.empty((H, W)) if return_y else None
    trace = np.full(max(max_iters, 1), np.nan)
    it = ctypes.c_int(0)
    st = lib.tvo_tv2d_pd(H, W, _p(f), _p(_f64(w_h)), _p(_f64(w_v)), float(lam), _p(_f64(y0)),
                         int(max_iters), float(tol), float(tau0), int(nthreads), _p(x),
                         ctypes.byref(it), _p(trace), _p(y))
    if st not in (0, 3):
        raise RuntimeError(f"oracle tv2d failed: {st}")
    out = (x, int(it.value), trace[:int(it.value)], st == 0)
    return out + (y,) if return_y else out


def tv2d_lagrangian(f, lam=0.0, w_h=None, w_v=None, tau0=100.0, max_iters=500, tol=1e-4,
                    check_every=5, nthreads=None):
    """ROF by the symmetric Lagrangian split of Sec. 6 (x_h, x_v, y) with tau_k = tau0 / k.

    Returns ``(x, iters, gap_trace, converged)``; ``gap_trace[k-1]`` is the per-pixel
    gap after iteration k where it was checked (NaN elsewhere).
    """
    lib = _load()
    f = _f64(f)
    H, W = f.shape
    nthreads = nthreads or os.cpu_count() or 1
    x = np.empty((H, W))
    trace = np.full(max_iters, np.nan)
    it = ctypes.c_int(0)
    st = lib.tvo_tv2d_lagrangian(H, W, _p(f), _p(_f64(w_h)), _p(_f64(w_v)), float(lam),
                                 float(tau0), int(max_iters), float(tol), int(check_every),
                                 int(nthreads), _p(x), ctypes.byref(it), _p(trace))
    if st not in (0, 3):
        raise RuntimeError(f"oracle tv2d_lagrangian failed: {st}")
    return x, int(it.value), trace[:int(it.value)], st == 0


def chain_solve_pq(a, b, alpha, f, w, offsets=None):
    """Chains with piecewise-quadratic unaries a_i x^2/2 - b_i x + alpha_i |x - f_i| and TV
    weights w (Sec. 4.2): one entry per node (w at a chain's last node unused); CSR
    ``offsets`` (default: one chain)."""
    a, b, alpha, f, w = (_f64(v) for v in (a, b, alpha, f, w))
    n = b.size
    if offsets is None:
        offsets = np.array([0, n], dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    x = np.empty(n, dtype=np.float64)
    st = _load().tvo_chain_solve_pq_batch(_p(a), _p(b), _p(alpha), _p(f), _p(w),
                                          offsets.ctypes.data_as(_I64), offsets.size - 1, _p(x))
    if st != 0:
        raise ValueError(f"oracle piecewise-quadratic chain solve failed ({st})")
    return x


def tv2d_l1(f, lam=0.0, w_h=None, w_v=None, tau=1.0, iters=100, nthreads=None):
    """TV-l1 denoising, min TV(x) + ||x - f||_1, by the primal-dual iteration with row
    chains of piecewise-quadratic unaries and column chains (constant steps, tau sigma = 1).
    Returns ``(x, energies)``; ``energies[k]`` is TV(x^{k+1}) + ||x^{k+1} - f||_1."""
    lib = _load()
    f = _f64(f)
    H, W = f.shape
    x = np.empty((H, W))
    e = np.empty(iters)
    st = lib.tvo_tv2d_l1(H, W, _p(f), _p(_f64(w_h)), _p(_f64(w_v)), float(lam), float(tau),
                         int(iters), int(nthreads or os.cpu_count() or 1), _p(x), _p(e))
    if st != 0:
        raise RuntimeError(f"oracle tv2d_l1 failed: {st}")
    return x, e


def chain_solve_nonconvex(unaries, w, C=None, offsets=None):
    """Chains with continuous piecewise-linear unaries and truncated TV (Sec. 3):
    min sum_i f_i(x_i) + sum_{i<n} min(w_i |x_{i+1} - x_i|, C_i).

    ``unaries``: one ``(lam, val, s_left, s_right)`` per node (breakpoints, values there,
    end slopes; s_left <= 0 <= s_right), or a tuple ``(uo, ul, uv, sl, sr)`` of CSR arrays.
    ``w``, ``C``: per node (edge to the next node; the last entry of a chain unused); C
    None or inf entries for plain TV. Returns ``(x, energies)`` with one optimum energy per
    chain."""
    if isinstance(unaries, tuple) and len(unaries) == 5:
        uo, ul, uv, sl, sr = unaries
        uo = np.ascontiguousarray(uo, dtype=np.int64)
        ul, uv, sl, sr = (_f64(a) for a in (ul, uv, sl, sr))
    else:
        lens = [len(u[0]) for u in unaries]
        uo = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        ul = _f64(np.concatenate([np.asarray(u[0], dtype=np.float64) for u in unaries]) if lens else [])
        uv = _f64(np.concatenate([np.asarray(u[1], dtype=np.float64) for u in unaries]) if lens else [])
        sl = _f64([u[2] for u in unaries])
        sr = _f64([u[3] for u in unaries])
    n = uo.size - 1
    w = _f64(w)
    C = np.full(n, np.inf) if C is None else _f64(C)
    if offsets is None:
        offsets = np.array([0, n], dtype=np.int64)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    x = np.empty(n, dtype=np.float64)
    e = np.empty(offsets.size - 1, dtype=np.float64)
    if ul.size == 0:
        ul = np.zeros(1)
        uv = np.zeros(1)
    st = _load().tvo_chain_solve_nonconvex_batch(uo.ctypes.data_as(_I64), _p(ul), _p(uv), _p(sl),
                                                 _p(sr), _p(w), _p(C),
                                                 offsets.ctypes.data_as(_I64), offsets.size - 1,
                                                 _p(x), _p(e))
    if st != 0:
        raise ValueError(f"oracle non-convex chain solve failed ({st})")
    return x, e
