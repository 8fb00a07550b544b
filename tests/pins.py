"""Independent checks that pin the oracle (and, on the GPU, the CUDA path).

Nothing here runs the paper's message-passing algorithm: each function follows
from the optimality conditions of eq. 1D-ROF / the ROF model, or calls a
library least-squares routine on the dual problem.

Optimality conditions used throughout (subgradient of the energy eq. main with
quadratic unaries and f_ij = w|z|): with u_0 = 0 and
u_e = sum_{k<=e} (x_k - c_k), a point x is the minimiser iff u_n = 0,
|u_e| <= w_e on every edge, and u_e = w_e * sign(x_{e+1} - x_e) where x jumps.
"""
from __future__ import annotations

import itertools

import numpy as np


def kkt_residual(c, w, x):
    """Largest violation of the chain optimality conditions (0 for the exact minimiser)."""
    c = np.asarray(c, np.float64)
    x = np.asarray(x, np.float64)
    w = np.broadcast_to(np.asarray(w, np.float64), (max(len(c) - 1, 0),))
    if len(c) == 0:
        return 0.0
    u = np.cumsum(x - c)
    viol = abs(u[-1])
    ue = u[:-1]
    if len(ue):
        viol = max(viol, float(np.max(np.abs(ue) - w, initial=0.0)))
        d = np.diff(x)
        jump = d != 0.0
        if np.any(jump):
            viol = max(viol, float(np.max(np.abs(ue[jump] - w[jump] * np.sign(d[jump])))))
    return viol


def brute_force_chain(c, w, tol=1e-12):
    """Exact minimiser of eq. 1D-ROF for short chains by enumerating, per edge,
    whether it is fused, a jump up or a jump down (3^(n-1) patterns).

    For a pattern the conditions fix u = +-w on jump edges, and each maximal
    fused run S = [l..r] gets x_S = mean(c_S) + (u_r - u_{l-1}) / |S|. The
    pattern is accepted when the jumps have the assumed signs and every fused
    edge satisfies |u_e| <= w_e. Returns the x of the first accepted pattern and
    checks that every accepted pattern gives the same x.
    """
    c = np.asarray(c, np.float64)
    n = len(c)
    w = np.broadcast_to(np.asarray(w, np.float64), (max(n - 1, 0),))
    if n == 1:
        return c.copy()
    found = None
    for pat in itertools.product((0, 1, -1), repeat=n - 1):
        u = np.zeros(n + 1)  # u[e+1] for edge e; u[0] = u[n] = 0
        for e, s in enumerate(pat):
            if s != 0:
                u[e + 1] = s * w[e]
        x = np.empty(n)
        l = 0
        while l < n:
            r = l
            while r < n - 1 and pat[r] == 0:
                r += 1
            seg = slice(l, r + 1)
            x[seg] = c[seg].mean() + (u[r + 1] - u[l]) / (r - l + 1)
            # fused edges inside the run: u from the running sum
            acc = u[l]
            for e in range(l, r):
                acc += x[e] - c[e]
                if abs(acc) > w[e] + tol:
                    break
            else:
                l = r + 1
                continue
            x = None
            break
        if x is None:
            continue
        ok = all((s == 0) or (s * (x[e + 1] - x[e]) >= -tol) for e, s in enumerate(pat))
        if not ok:
            continue
        if found is None:
            found = x
        else:
            assert np.allclose(found, x, atol=1e-9), "two optimality patterns disagree"
    assert found is not None, "no pattern satisfies the optimality conditions"
    return found


def bvls_chain(c, w):
    """Minimiser of eq. 1D-ROF through its dual, a box-constrained least-squares
    problem min_u ||c - D^T u|| s.t. |u| <= w solved by scipy's BVLS; x = c - D^T u."""
    from scipy.optimize import lsq_linear

    c = np.asarray(c, np.float64)
    n = len(c)
    if n == 1:
        return c.copy()
    w = np.broadcast_to(np.asarray(w, np.float64), (n - 1,)).copy()
    D = np.zeros((n - 1, n))
    D[np.arange(n - 1), np.arange(n - 1)] = -1.0
    D[np.arange(n - 1), np.arange(1, n)] = 1.0
    free = w > 0
    u = np.zeros(n - 1)
    if np.any(free):
        res = lsq_linear(D[free].T, c, bounds=(-w[free], w[free]), method="bvls", tol=1e-15)
        u[free] = res.x
    return c - D.T @ u


def rof_exact(f, w_h, w_v):
    """Minimiser of the 2D ROF model of Sec. 6.1 on a small image through its dual
    min_p ||f - D_h^T p_h - D_v^T p_v|| s.t. |p| <= w (scipy BVLS); x = f - D^T p."""
    from scipy.optimize import lsq_linear

    f = np.asarray(f, np.float64)
    H, W = f.shape
    idx = np.arange(H * W).reshape(H, W)
    pairs = [(idx[:, :-1].ravel(), idx[:, 1:].ravel(), np.asarray(w_h, np.float64).ravel()),
             (idx[:-1, :].ravel(), idx[1:, :].ravel(), np.asarray(w_v, np.float64).ravel())]
    m = sum(len(p[0]) for p in pairs)
    D = np.zeros((m, H * W))
    bnd = np.zeros(m)
    r = 0
    for a, b, ww in pairs:
        k = len(a)
        D[np.arange(r, r + k), a] = -1.0
        D[np.arange(r, r + k), b] = 1.0
        bnd[r:r + k] = ww
        r += k
    res = lsq_linear(D.T, f.ravel(), bounds=(-bnd, bnd), method="bvls", tol=1e-15,
                     max_iter=200000)
    return (f.ravel() - D.T @ res.x).reshape(H, W)


def read_closed_forms(path):
    """Parse the hand-derived fixtures: ``c ; w ; x ; note`` per line."""
    cases = []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = [p.strip() for p in line.split(";")]
        c = np.array([float(v) for v in parts[0].split()])
        w = np.array([float(v) for v in parts[1].split()]) if parts[1] else np.zeros(0)
        x = np.array([float(v) for v in parts[2].split()])
        cases.append((c, w, x, parts[3] if len(parts) > 3 else ""))
    return cases
