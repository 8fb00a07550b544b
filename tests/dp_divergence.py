"""Loop statistics of the one-thread-per-chain-half message update, on the host.

The thread form of the chain DP (Algorithm 2, updates of Sec. 4.1) removes breakpoints
from the ends of a message in two data-dependent scans per node, plus a short re-walk
from the other end when a scan removed more than half of the message. In a warp the
32 lanes (16 chains, two halves each, rooted at the middle node) run these loops in
lockstep, so every node step costs the warp the longest loop among its lanes.

This module replays exactly that control flow in FP32 on the host (no GPU, no device
code) and counts, per node step, the iterations of each loop for every lane and the
maximum over the warp. The ratio between the two is the SIMT divergence that bounds
the thread kernel's instruction count.

    python -m tests.dp_divergence [--chains 64] [--len 1024] [--lam 0.15]
"""
from __future__ import annotations

import argparse

import numpy as np

from paper_1502_07770_gb300 import synth

f32 = np.float32


def half_loops(c, lam, records=None):
    """Iterations of (left scan, left re-walk, right scan, right re-walk) and the message
    size after every update of one half, whose nodes in walk order have unaries c.
    ``lam`` is the weight of every node's edge towards the root, or a sequence of them.
    With ``records`` (a list), the (lambda-, lambda+) of every node is appended to it."""
    ws = np.broadcast_to(np.asarray(lam, dtype=np.float32), (len(c),))
    ring = {}
    out = []
    if len(c) == 0:
        return np.zeros((0, 5), dtype=np.int64)
    c0, lam = f32(c[0]), f32(ws[0])
    fl, fs, bl, bs, wprev = c0 - lam, f32(0), c0 + lam, f32(-1), lam
    if records is not None:
        records.append((fl, bl))
    F, B = 0, 1
    ring[F], ring[B] = (fl, fs), (bl, bs)
    for i in range(1, len(c)):
        ci, wi, abar = f32(c[i]), f32(ws[i]), f32(i + 1)
        nwi = -wi
        vF = fl - ci - wprev
        al, av, asl, as_ = fl, vF, f32(1), f32(1) - abar
        lastL, p, pl, ps, v = F - 1, F, fl, fs, vF
        itL = wL = itR = wR = 0
        while v < nwi:
            itL += 1
            al, av, asl, as_, lastL = pl, v, ps + abar, ps, p
            if p == B:
                break
            ql, qs = ring[p + 1]
            v = f32(v + asl * (ql - pl))
            p, pl, ps = p + 1, ql, qs
        if lastL - F > B - lastL:
            vb, ql = bl - ci + wprev, bl
            for q in range(B - 1, lastL - 1, -1):
                el, es = ring[q]
                vb = f32(vb - (es + abar) * (ql - el))
                ql = el
                wL += 1
            av = vb
        lm, lm_s = f32(al + (nwi - av) / asl), as_
        bl2, bv, bsl = bl, bl - ci + wprev, f32(1)
        lastR, from_lm = B + 1, B <= lastL
        if not from_lm:
            q, ql, v = B, bl, bv
            while v > wi:
                itR += 1
                lastR = q
                if q - 1 <= lastL:
                    from_lm = True
                    break
                el, es = ring[q - 1]
                sl = es + abar
                bl2, bv, bsl = ql, v, sl
                v = f32(v - sl * (ql - el))
                q, ql = q - 1, el
            if not from_lm and lastR <= B and B - lastR > lastR - F:
                vf, el, es = vF, fl, fs
                for t in range(F + 1, lastR + 1):
                    e2l, e2s = ring[t]
                    vf = f32(vf + (es + abar) * (e2l - el))
                    el, es = e2l, e2s
                    wR += 1
                bv = vf
        if from_lm:
            bl2, bv, bsl = lm, nwi, lm_s + abar
        hp = f32(bl2 + (wi - bv) / bsl)
        if records is not None:
            records.append((lm, hp))
        nF = lastL
        nB = max(lastR - 1, nF) + 1
        ring[nF], ring[nB] = (lm, lm_s), (hp, -abar)
        F, B, fl, fs, bl, bs, wprev = nF, nB, lm, lm_s, hp, -abar, wi
        out.append((itL, wL, itR, wR, B - F + 1))
    return np.asarray(out, dtype=np.int64)


def replay_chain(y, lam):
    """The whole chain solved by the replayed update from node 0 (weight lam on every edge,
    0 on the virtual edge after the last node) and the backward clips of Algorithm 2; used
    to check the replay against an independent solver."""
    n = len(y)
    if n == 1:
        return np.array([y[0]], dtype=np.float64)
    w = np.full(n, lam, dtype=np.float32)
    w[-1] = 0.0
    rec = []
    half_loops(np.asarray(y, np.float32), w, records=rec)
    x = np.empty(n)
    x[-1] = 0.5 * (float(rec[-1][0]) + float(rec[-1][1]))
    for i in range(n - 2, -1, -1):
        x[i] = min(max(x[i + 1], float(rec[i][0])), float(rec[i][1]))
    return x


def warp_stats(y, lam):
    """Statistics over warps of 16 chains (rows of y, all of one length)."""
    n = y.shape[1]
    mid = n // 2
    lane_sum = np.zeros(4)
    warp_sum = np.zeros(4)
    sizes = []
    steps = 0
    lane_steps = 0
    for g in range(y.shape[0] // 16):
        per = []
        for k in range(16 * g, 16 * g + 16):
            per.append(half_loops(y[k, :mid], lam))            # nodes 0 .. mid-1
            per.append(half_loops(y[k, mid + 1:][::-1], lam))  # nodes n-1 .. mid+1
        T = max(len(a) for a in per)
        A = np.zeros((len(per), T, 5), dtype=np.int64)
        for l, a in enumerate(per):
            A[l, :len(a)] = a
        lane_sum += A[:, :, :4].sum(axis=(0, 1))
        lane_steps += sum(len(a) for a in per)
        warp_sum += A[:, :, :4].max(axis=0).sum(axis=0)
        steps += T
        sizes.append(A[:, :, 4].ravel())
    s = np.concatenate(sizes)
    return {"lane_mean": lane_sum / lane_steps, "warp_max": warp_sum / steps,
            "size_mean": float(s[s > 0].mean()), "size_max": int(s.max())}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--chains", type=int, default=64)
    ap.add_argument("--len", type=int, default=1024)
    ap.add_argument("--lam", type=float, default=0.15)
    a = ap.parse_args(argv)
    y = synth.chain_batch(a.chains, a.len, seed0=1000)
    r = warp_stats(y, a.lam)
    names = ("left scan", "left re-walk", "right scan", "right re-walk")
    print(f"{a.chains} chains x {a.len} nodes, lambda {a.lam}; per node step:")
    print(f"{'loop':<14} {'lane mean':>10} {'warp max':>10}")
    for nm, m, w in zip(names, r["lane_mean"], r["warp_max"]):
        print(f"{nm:<14} {m:10.3f} {w:10.3f}")
    print(f"{'total':<14} {r['lane_mean'].sum():10.3f} {r['warp_max'].sum():10.3f}")
    print(f"message size: mean {r['size_mean']:.2f}, max {r['size_max']}")


if __name__ == "__main__":
    main()
