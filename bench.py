#!/usr/bin/env python
"""Benchmark of the GB300 TV library.

Headline: milliseconds per 1024x1024 2D TV-l2 (ROF) denoise to per-pixel
primal-dual gap 1e-4 (Lagrangian decomposition, eq. pd, row/column chain
proxes), on the synthetic image of 200 random rectangles and disks plus
Gaussian noise 0.1, lambda 0.1. One step = one full denoise from the call to
the returned result, inputs resident in HBM; L2 is flushed (a 256 MB write)
before every step, outside the timed span.

Also reported: batched chain-prox throughput (Gnode/s) on 65536 chains of
1024 nodes, the roofline of the dominant kernel, SM clocks sampled during the
timed region, an end-to-end number through host buffers, and the FP64 CPU
oracle timed on a bounded sample on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run: every rank denoises its own copy
(independent replicas, no collective on the data path).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gnode/s batched chain-TV prox; ms per 1024² 2D-TV denoise to gap 1e-4"
H = W = 1024
LAM = 0.1
TOL = 1e-4
MAX_ITERS = 200
CHAIN_B, CHAIN_N, CHAIN_LAM = 65536, 1024, 0.15
CFG0_B, CFG0_N, CFG0_LAM = 512, 256, 0.2
L2_FLUSH_BYTES = 256 << 20
WORKLOAD = ("ROF denoise 1024x1024 (200 rectangles/disks, levels U[0,1], + N(0,0.1^2)), "
            "lambda 0.1, 4-connected, tau0=sigma0=1, to per-pixel gap 1e-4")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="bounded CPU work for the oracle baseline")
    return ap.parse_args()


LEARNED_EVAL = 24


def npx_net(h, w):
    """Multiply-adds of one network inference on an h x w image (3x3 convs 16->32->32->32->16)."""
    return h * w * 9 * (16 * 32 + 32 * 32 + 32 * 32 + 32 * 16)


def peaks_bf16():
    """Measured dense BF16 tensor peak (TFLOP/s, burst) and where it came from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            m = json.load(fh)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources each recorded kernel is built from (its translation unit and the
# shared headers): a change to any of them voids that kernel's recorded traffic
KERNEL_SOURCES = {
    "tv2d": ["tv2d.cu", "tv2d_common.cuh", "tv_coop.cuh", "tv_dp.cuh", "tv_launch.cuh", "tv_host.h"],
    "chain": ["tv_chain.cu", "tv_flat.cuh", "tv_halves.cuh", "tv_coop.cuh", "tv_dp.cuh", "tv_launch.cuh",
              "tv_host.h"],
    "pq": ["tv_pq.cu", "tv_coop.cuh", "tv_dp.cuh", "tv_launch.cuh", "tv_host.h"],
}


def kernel_source_hash(group):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1502_07770_gb300", "csrc")
    for f in KERNEL_SOURCES[group]:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kind):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current sources of that kernel; else None."""
    group = kind.split("_")[0]
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
        if t.get("source_hash", {}).get(group) == kernel_source_hash(group):
            return t.get(kind)
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampler (SM clock, max clock, throttle reasons) around the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _timed_runs(fn, seconds, min_runs=1):
    """Runs fn() until `seconds` of wall time have passed (at least min_runs times);
    returns (runs, elapsed seconds, last result)."""
    runs, t0, r = 0, time.perf_counter(), None
    while True:
        r = fn()
        runs += 1
        el = time.perf_counter() - t0
        if el >= seconds and runs >= min_runs:
            return runs, el, r


def cpu_baseline(f, seconds, chain_y, chain_lam):
    """The FP64 oracle (as it stands) on the host cores, on bounded samples: repeated
    full 1024x1024 denoises until `seconds` of wall time have passed, on all cores and on
    one thread (the paper's single-core regime); and the batched chain prox (Gnode/s) on
    a block of the benchmark's chains, on all cores and on one thread."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.build()

    def denoise(nt):
        return oracle.tv2d_pd(f, lam=LAM, max_iters=MAX_ITERS, tol=TOL, nthreads=nt)[1]
    runs, el, iters = _timed_runs(lambda: denoise(threads), seconds, 2)
    ms = el / runs * 1e3
    runs1, el1, _ = _timed_runs(lambda: denoise(1), seconds / 2, 1)
    ms1 = el1 / runs1 * 1e3
    nb, nn = chain_y.shape
    flat = chain_y.reshape(-1)
    offs = np.arange(nb + 1, dtype=np.int64) * nn

    def chains(nt):
        return oracle.chain_solve_batch(flat, offs, lam=chain_lam, nthreads=nt)
    cr, cel, _ = _timed_runs(lambda: chains(threads), seconds / 4, 2)
    cr1, cel1, _ = _timed_runs(lambda: chains(1), seconds / 4, 1)
    return {"value": ms, "unit": "ms", "cores": threads, "kind": "oracle",
            "cpu_model": cpu_model(),
            "sample": f"{runs} full 1024x1024 denoises ({iters} iterations each), FP64, "
                      f"{threads} threads, {el:.1f} s",
            "single_thread": {"value": ms1, "unit": "ms", "cores": 1,
                              "sample": f"{runs1} full denoises on one thread, {el1:.1f} s"},
            "chain_prox": {"value": nb * nn * cr / cel / 1e9, "unit": "Gnode/s", "cores": threads,
                           "single_thread": nb * nn * cr1 / cel1 / 1e9,
                           "sample": f"{nb} chains x {nn} nodes of the chain-prox workload, "
                                     f"lambda {chain_lam}, FP64; {cr} runs on {threads} threads "
                                     f"({cel:.1f} s), {cr1} on one ({cel1:.1f} s)"}}


def max_over_ranks(value, device, world):
    """The largest of each rank's value (the job's time is its slowest rank's); the value
    itself with one rank. Uses the initialised default process group."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on the same workload, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1502_07770_gb300 import synth
    import oracle
    oracle.build()
    _, f = synth.shapes_image(H, W, seed=0)
    threads = os.cpu_count() or 1
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.tv2d_pd(f, lam=LAM, max_iters=MAX_ITERS, tol=TOL, nthreads=threads)
    ts = []
    iters = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, iters, _, _ = oracle.tv2d_pd(f, lam=LAM, max_iters=MAX_ITERS, tol=TOL, nthreads=threads)
        ts.append((time.perf_counter() - t0) * 1e3)
    ms = float(np.mean(ts))
    out = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "iterations": iters},
           "cpu_baseline": {"value": ms, "unit": "ms", "cores": threads, "kind": "oracle",
                            "cpu_model": cpu_model(),
                            "sample": f"{args.steps} full denoises, {threads} threads"},
           "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_1502_07770_gb300 import _lib, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    _lib.load()
    _, f_np = synth.shapes_image(H, W, seed=0)
    f = torch.from_numpy(f_np).to(dev)
    x = torch.empty_like(f)
    ws = _lib.workspace(_lib.load().tv2d_workspace_size(H, W, MAX_ITERS), dev, "bench2d")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return _lib.tv2d_denoise(f, lam=LAM, max_iters=MAX_ITERS, tol=TOL, out=x, ws=ws)

    for _ in range(args.warmup):
        flush.zero_()
        r = step()
    iters, gap, ok = r[1], r[2], r[3]
    if not ok:
        raise RuntimeError(f"denoise did not converge: {iters} iterations, gap {gap}")

    # ---------------- timed region: K denoises ----------------
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    _lib.profile_enable(False)
    barrier()
    launches0 = _lib.launch_count()
    step_ms = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
    barrier()
    launches = _lib.launch_count() - launches0
    clk = clocks.stop()

    # Per-phase launch durations: the same K steps again with the library's CUDA events
    # around every phase launch. The event records add host work between launches, so
    # they stay out of the timed steps above.
    _lib.profile_enable(True)
    for kind in ("col", "row", "init", "chain"):
        _lib.profile_read(kind)
    for _ in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize(dev)
    prof = {k: _lib.profile_read(k) for k in ("col", "row", "init")}
    _lib.profile_enable(False)
    ms_step = float(np.sum(step_ms)) / args.steps
    ms_step = max_over_ranks(ms_step, dev, world)

    # ---------------- end to end through host buffers ----------------
    h_in = torch.from_numpy(f_np).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d_in = torch.empty_like(f)
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        d_in.copy_(h_in, non_blocking=True)
        _lib.tv2d_denoise(d_in, lam=LAM, max_iters=MAX_ITERS, tol=TOL, out=x, ws=ws)
        h_out.copy_(x, non_blocking=True)
        torch.cuda.synchronize(dev)
        if it >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = float(np.mean(e2e_ms))
    e2e = max_over_ranks(e2e, dev, world)

    # ---------------- batched chain prox (Gnode/s) ----------------
    base = synth.chain_batch(256, CHAIN_N, seed0=1000)
    yc = torch.from_numpy(np.tile(base, (CHAIN_B // 256, 1))).to(dev)
    xc = torch.empty_like(yc)
    wsc = _lib.workspace(_lib.load().tv_chain_workspace_size(CHAIN_B, CHAIN_N), dev, "benchchain")
    for _ in range(3):
        _lib.chain_prox(yc, lam=CHAIN_LAM, out=xc, ws=wsc)
    _lib.profile_enable(True)
    _lib.profile_read("chain")
    chain_ms = []
    for _ in range(max(5, args.steps // 5)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.chain_prox(yc, lam=CHAIN_LAM, out=xc, ws=wsc)
        b.record(stream)
        b.synchronize()
        chain_ms.append(a.elapsed_time(b))
    kms, kn = _lib.profile_read("chain")
    _lib.profile_enable(False)
    st, overflowed = _lib.workspace_status(wsc)
    nodes = CHAIN_B * CHAIN_N
    cms = float(np.median(chain_ms))
    hbm, peak_kind = peaks()
    chain_kernel_ms = kms / max(kn, 1)
    chain_achieved = 8.0 * nodes / (chain_kernel_ms * 1e-3) / 1e9

    # ---------------- the 512 x 256 chain batch (launch-bound: 1 MB of traffic) ----------
    y0c = torch.from_numpy(synth.chain_batch(CFG0_B, CFG0_N, seed0=0)).to(dev)
    x0c = torch.empty_like(y0c)
    ws0 = _lib.workspace(_lib.load().tv_chain_workspace_size(CFG0_B, CFG0_N), dev, "benchcfg0")
    for _ in range(3):
        _lib.chain_prox(y0c, lam=CFG0_LAM, out=x0c, ws=ws0)
    cfg0_ms = []
    for _ in range(max(10, args.steps // 2)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.chain_prox(y0c, lam=CFG0_LAM, out=x0c, ws=ws0)
        b.record(stream)
        b.synchronize()
        cfg0_ms.append(a.elapsed_time(b))
    c0ms = float(np.median(cfg0_ms))
    cfg0 = {"value": CFG0_B * CFG0_N / (c0ms * 1e-3) / 1e9, "unit": "Gnode/s", "ms": c0ms,
            "workload": f"{CFG0_B} chains x {CFG0_N} nodes (seeds 0..{CFG0_B - 1}), lambda "
                        f"{CFG0_LAM}, piecewise-constant + N(0,0.1^2), L2 flushed",
            "note": "1.05 MB of algorithmic traffic: bound by launch and the sequential "
                    "256-node chains, not by HBM"}
    del y0c, x0c

    # ---------------- chain-prox sweep: shapes and per-edge weights ----------------
    sweep = []
    for SB, SN in ((65536, 1024), (262144, 256), (16384, 4096)):
        sbase = synth.chain_batch(256, SN, seed0=2000)
        ys = torch.from_numpy(np.tile(sbase, (SB // 256, 1))).to(dev)
        xs = torch.empty_like(ys)
        wsw = _lib.workspace(_lib.load().tv_chain_workspace_size(SB, SN), dev, "benchsweep")
        for weighted in (False, True):
            wt = None
            if weighted:
                wrow = np.random.default_rng(3).uniform(0.05, 0.3, size=(256, SN)).astype(np.float32)
                wt = torch.from_numpy(np.tile(wrow, (SB // 256, 1))).to(dev)
            for _ in range(2):
                _lib.chain_prox(ys, wt, lam=CHAIN_LAM, out=xs, ws=wsw)
            tms = []
            for _ in range(5):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                _lib.chain_prox(ys, wt, lam=CHAIN_LAM, out=xs, ws=wsw)
                b.record(stream)
                b.synchronize()
                tms.append(a.elapsed_time(b))
            t = float(np.median(tms))
            bpn = 12.0 if weighted else 8.0
            gbs = bpn * SB * SN / (t * 1e-3) / 1e9
            sweep.append({"chains": SB, "nodes": SN, "weights": "per-edge" if weighted else "uniform",
                          "ms": t, "Gnode_per_s": SB * SN / (t * 1e-3) / 1e9,
                          "bytes_per_node": bpn, "GB_per_s": gbs, "frac": gbs / peaks()[0]})
            del wt
        del ys, xs

    # ---------------- general convex chains (curvature a_i, slopes w^-_i <= w^+_i) ----------
    GB, GN = 2048, 1024
    grng = np.random.default_rng(11)
    ga = grng.uniform(0.5, 2.0, (GB, GN)).astype(np.float32)
    gb = (ga * np.tile(synth.chain_batch(256, GN, seed0=3000), (GB // 256, 1))).astype(np.float32)
    gwl = grng.uniform(-0.3, 0.05, (GB, GN)).astype(np.float32)
    gwh = (gwl + grng.uniform(0.0, 0.4, (GB, GN))).astype(np.float32)
    gt = [torch.from_numpy(v).to(dev) for v in (ga, gb, gwl, gwh)]
    gx = torch.empty_like(gt[1])
    for _ in range(3):
        _lib.chain_prox_general(gt[1], gt[2], gt[3], a=gt[0], out=gx)
    gms = []
    for _ in range(10):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.chain_prox_general(gt[1], gt[2], gt[3], a=gt[0], out=gx)
        b.record(stream)
        b.synchronize()
        gms.append(a.elapsed_time(b))
    gmed = float(np.median(gms))
    general = {"value": GB * GN / (gmed * 1e-3) / 1e9, "unit": "Gnode/s", "ms": gmed,
               "workload": f"{GB} chains x {GN}, a ~ U[0.5,2], b = a * (step signal), "
                           "w^- ~ U[-0.3,0.05], w^+ = w^- + U[0,0.4]",
               "bytes_per_node": 20,
               "GB_per_s": 20.0 * GB * GN / (gmed * 1e-3) / 1e9}
    del gt, gx

    # ---------------- differentiable prox: forward + backward ----------------
    DB, DN = 4096, 1024
    yd = torch.from_numpy(synth.chain_batch(DB, DN, seed0=1000)).to(dev)
    cd = torch.from_numpy(synth.gaussian_vector(DB * DN, seed=7).reshape(DB, DN)).to(dev)
    xd = torch.empty_like(yd)
    wsd = _lib.workspace(_lib.load().tv_chain_workspace_size(DB, DN), dev, "benchdiff")
    for _ in range(3):
        _lib.chain_prox(yd, lam=0.15, out=xd, ws=wsd)
        _lib.chain_prox_backward(xd, cd)
    _lib.profile_enable(True)
    _lib.profile_read("grad")
    diff_ms = []
    for _ in range(max(5, args.steps // 5)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.chain_prox(yd, lam=0.15, out=xd, ws=wsd)
        _lib.chain_prox_backward(xd, cd)
        b.record(stream)
        b.synchronize()
        diff_ms.append(a.elapsed_time(b))
    gms, gn = _lib.profile_read("grad")
    _lib.profile_enable(False)
    grad_kernel_ms = gms / max(gn, 1)
    grad_achieved = 12.0 * DB * DN / (grad_kernel_ms * 1e-3) / 1e9
    dms = float(np.median(diff_ms))

    # ---------------- batched uneven images (64 images, 128x96 .. 2048x1536) ----------------
    sizes, blams = synth.uneven_image_sizes(64, seed=100)
    bfs = [synth.shapes_image(h, w, seed=100 + m)[1] for m, (h, w) in enumerate(sizes)]
    bws = [synth.edge_aware_weights(fm, blams[m]) for m, fm in enumerate(bfs)]
    bimg = [torch.from_numpy(fm).to(dev) for fm in bfs]
    bwh = [torch.from_numpy(w[0]).to(dev) for w in bws]
    bwv = [torch.from_numpy(w[1]).to(dev) for w in bws]
    bouts = [torch.empty_like(t) for t in bimg]
    bpix = sum(h * w for h, w in sizes)

    def batched():
        return _lib.tv2d_denoise_batched(bimg, blams, bwh, bwv, max_iters=MAX_ITERS, tol=TOL,
                                         outs=bouts)
    r = batched()
    b_iters = r[1]
    # algorithmic bytes: per image and iteration 40 B a pixel (column phase: read x^k,
    # x^{k-1}, y, w_v, write y; row phase: read f, x^k, y, w_h, write x^{k+1}); an image
    # stops at its own iteration count
    b_bytes = 40.0 * sum(h * w * int(k) for (h, w), k in zip(sizes, b_iters))
    batched_ms = []
    for _ in range(max(3, args.steps // 10)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        batched()
        b.record(stream)
        b.synchronize()
        batched_ms.append(a.elapsed_time(b))
    bms = float(np.median(batched_ms))
    # the same images one call each (the plain method, image by image)
    seq_ms = []
    for _ in range(max(2, args.steps // 25)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for m in range(len(bimg)):
            _lib.tv2d_denoise(bimg[m], lam=blams[m], w_h=bwh[m], w_v=bwv[m], max_iters=MAX_ITERS,
                              tol=TOL, out=bouts[m])
        b.record(stream)
        b.synchronize()
        seq_ms.append(a.elapsed_time(b))
    sms = float(np.median(seq_ms))

    # ---------------- the symmetric Lagrangian split on the same image ----------------
    lag_ms = []
    for rep in range(args.warmup + max(3, args.steps // 10)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rl = _lib.tv2d_denoise_lagrangian(f, lam=LAM, tau0=10.0, max_iters=1000, tol=TOL,
                                          check_every=5, out=x)
        b.record(stream)
        b.synchronize()
        if rep >= args.warmup:
            lag_ms.append(a.elapsed_time(b))
    lagrangian = {"ms": float(np.median(lag_ms)), "iterations": rl[1], "gap": rl[2],
                  "converged": bool(rl[3]), "tau0": 10.0, "check_every": 5,
                  "workload": "the 1024x1024 image of the headline, lambda 0.1, per-pixel gap "
                              "1e-4 (P(xbar) - D(y), Lagrangian dual)"}

    # ---------------- TV-l1 denoising (Sec. 6) on an impulse-noise image ----------------
    f1 = torch.from_numpy(synth.salt_pepper_image(H, W, seed=7)).to(dev)
    L1_ITERS = 100
    l1_ms = []
    for rep in range(args.warmup + max(3, args.steps // 10)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r1 = _lib.tv2d_denoise_l1(f1, lam=0.55, tau=0.1, max_iters=L1_ITERS, tol=0.0,
                                  check_every=L1_ITERS, out=x)
        b.record(stream)
        b.synchronize()
        if rep >= args.warmup:
            l1_ms.append(a.elapsed_time(b))
    _lib.profile_enable(True)
    _lib.profile_read("col")
    _lib.profile_read("row")
    _lib.tv2d_denoise_l1(f1, lam=0.55, tau=0.1, max_iters=L1_ITERS, tol=0.0,
                         check_every=L1_ITERS, out=x)
    torch.cuda.synchronize(dev)
    l1c, l1r = _lib.profile_read("col"), _lib.profile_read("row")
    _lib.profile_enable(False)
    pq_ms = l1r[0] / max(l1r[1], 1)
    pq_achieved = 12.0 * H * W / (pq_ms * 1e-3) / 1e9  # read xi, f; write x
    tv_l1 = {"ms": float(np.median(l1_ms)), "iterations": r1[1],
             "col_kernel_ms": l1c[0] / max(l1c[1], 1), "row_kernel_ms": pq_ms,
             "row_roofline": {"bound": "hbm", "kernel": "pq_halves_kernel", "achieved": pq_achieved,
                              "peak": hbm, "unit": "GB/s", "frac": pq_achieved / hbm,
                              "traffic": recorded_traffic("pq_row"), "bytes_per_pixel": 12},
             "ms_per_iteration": float(np.median(l1_ms)) / L1_ITERS, "energy": r1[2],
             "tau": 0.1, "workload": f"{H}x{W} shapes image with 25% salt-and-pepper pixels, "
                                     "lambda 0.55, 100 iterations of eq. pd (column chains + "
                                     "piecewise-quadratic row chains)"}

    # ---------------- non-convex chains (Sec. 3) on a stereo-sized cost volume ----------------
    NC_H, NC_W, NC_L = 1000, 1482, 126
    nc_cost = torch.from_numpy(synth.stereo_cost_volume(NC_H, NC_W, NC_L, seed=0)[0]).to(dev)
    nc_x = torch.empty(NC_H * NC_W, dtype=torch.float32, device=dev)
    nc_e = torch.empty(NC_H, dtype=torch.float64, device=dev)
    nc_ms = []
    for rep in range(args.warmup + max(3, args.steps // 10)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _lib.chain_prox_nonconvex(nc_cost, sl=-1.0, sr=1.0, w=0.1, C=0.8, max_breakpoints=512,
                                  out=nc_x, energy=nc_e)
        b.record(stream)
        b.synchronize()
        if rep >= args.warmup:
            nc_ms.append(a.elapsed_time(b))
    nc_status, _ = _lib.workspace_status(_lib.workspace(1, dev, "nonconvex"))
    ncm = float(np.median(nc_ms))
    nc_nodes = NC_H * NC_W
    nc_bytes = nc_nodes * (NC_L * 4 + 4)  # read the node's costs, write x
    nc_achieved = nc_bytes / (ncm * 1e-3) / 1e9
    nonconvex = {"ms": ncm, "value": nc_nodes / (ncm * 1e-3) / 1e9, "unit": "Gnode/s",
                 "status": int(nc_status), "max_breakpoints": 512,
                 "roofline": {"bound": "hbm", "kernel": "nc_chain_kernel", "achieved": nc_achieved,
                              "peak": hbm, "unit": "GB/s", "frac": nc_achieved / hbm,
                              "bytes_per_node": NC_L * 4 + 4,
                              "note": "latency-bound: one warp per chain, 1000 chains"},
                 "workload": f"{NC_H} chains x {NC_W} nodes, cost volume of {NC_L} disparities "
                             "(truncated-linear cost + noise + 10% false minima), w 0.1, C 0.8, "
                             "the size of the paper's stereo pair"}
    del nc_cost

    # ---------------- learned dual warm start (stored network) ----------------
    from paper_1502_07770_gb300 import learned
    net = learned.load_weights(dev)
    lsum, _ = learned.evaluate(net, range(20000, 20000 + LEARNED_EVAL), H=512, W=512, tol=TOL,
                               max_iters=MAX_ITERS, reps=3, device=dev)
    lam_t = torch.tensor([LAM], dtype=torch.float32, device=dev)
    warm_ms = []
    for rep in range(args.warmup + max(5, args.steps // 5)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rw = learned.denoise_warm(net, f, LAM, lam_t, tol=TOL, max_iters=MAX_ITERS)
        b.record(stream)
        b.synchronize()
        if rep >= args.warmup:
            warm_ms.append(a.elapsed_time(b))
    for _ in range(3):
        net.predict_dual(f, lam_t)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(10):
        net.predict_dual(f, lam_t)
    b.record(stream)
    b.synchronize()
    net_ms = a.elapsed_time(b) / 10
    net_flop = 2.0 * npx_net(H, W)
    bf16_peak = peaks_bf16()

    # ---------------- roofline of the dominant kernel of the step ----------------
    # algorithmic bytes: column (dual) phase reads x^k, x^{k-1}, y, f and writes y
    # (16 B/pixel); row (primal) phase reads f, x^k, y and writes x^{k+1} (16 B/pixel).
    # The library times only the launches that did work: the phases of iterations
    # launched after the stop flag was set return at once and are left out.
    npx = H * W
    dom = max(("col", "row"), key=lambda k: prof[k][0])
    dom_ms_total, dom_launches = prof[dom]
    dom_bytes = 16.0 * npx * dom_launches
    dom_achieved = dom_bytes / (dom_ms_total * 1e-3) / 1e9
    traffic = recorded_traffic(f"tv2d_{dom}")

    result = {
        "metric": METRIC,
        "value": ms_step / world,
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "iterations": iters, "gap": gap,
                   "l2": "flushed before every step (256 MB write, not timed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "e2e": {"value": e2e / world, "unit": "ms", "h2d_bytes_per_step": npx * 4,
                "d2h_bytes_per_step": npx * 4},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": f"tv2d {dom} phase", "achieved": dom_achieved,
                     "peak": hbm, "unit": "GB/s", "frac": dom_achieved / hbm,
                     "traffic": traffic, "peak_kind": peak_kind,
                     "bytes_per_launch": 16.0 * npx,
                     "avg_launch_ms": dom_ms_total / max(dom_launches, 1),
                     "note": "latency-bound: state of ~24 MB stays in L2; 1024 chains per phase"},
        "phase_ms_per_step": {k: prof[k][0] / args.steps for k in prof},
        "phase_launches_per_step": {k: prof[k][1] / args.steps for k in prof},
        "chain_prox": {"value": nodes / (cms * 1e-3) / 1e9, "unit": "Gnode/s",
                       "workload": f"{CHAIN_B} chains x {CHAIN_N} nodes, lambda {CHAIN_LAM}, "
                                   "piecewise-constant + N(0,0.1^2), L2 flushed",
                       "ms": cms, "overflowed_chains": int(overflowed),
                       "roofline": {"bound": "hbm", "achieved": chain_achieved, "peak": hbm,
                                    "unit": "GB/s", "frac": chain_achieved / hbm,
                                    "traffic": recorded_traffic("chain"),
                                    "bytes_per_node": 8}},
        "chain_prox_512x256": cfg0,
        "chain_prox_sweep": sweep,
        "general_chain": general,
        "diff_prox": {"value": DB * DN / (dms * 1e-3) / 1e9, "unit": "Gnode/s",
                      "workload": f"{DB} chains x {DN}, lambda 0.15, forward + backward "
                                  "(loss sum c_i x_i, c ~ N(0,1)), L2 flushed",
                      "ms": dms, "backward_kernel_ms": grad_kernel_ms,
                      "backward_roofline": {"bound": "hbm", "achieved": grad_achieved,
                                            "peak": hbm, "unit": "GB/s",
                                            "frac": grad_achieved / hbm, "bytes_per_node": 12}},
        "batched": {"ms": bms, "images": len(sizes), "megapixels": bpix / 1e6,
                    "Mpixel_per_s": bpix / (bms * 1e-3) / 1e6,
                    "iterations_max": int(max(b_iters)), "iterations_mean": float(np.mean(b_iters)),
                    "graph_loop": int(_lib.load().tv2d_batched_last_mode()),
                    "sequential_ms": sms,
                    "speedup_vs_sequential": sms / bms,
                    "roofline": {"bound": "hbm", "achieved": b_bytes / (bms * 1e-3) / 1e9,
                                 "peak": hbm, "unit": "GB/s",
                                 "frac": b_bytes / (bms * 1e-3) / 1e9 / hbm,
                                 "bytes_per_pixel_iteration": 40,
                                 "note": "whole solve (both phases, gap kernels, graph "
                                         "loop) over the summed per-image iterations"},
                    "workload": "64 images, W ~ U{128..2048}, H ~ U{96..1536}, lambda ~ U[0.05,0.3], "
                                "edge-aware weights lambda*exp(-|df|/0.2), to per-pixel gap 1e-4"},
        "lagrangian_split": lagrangian,
        "tv_l1": tv_l1,
        "nonconvex_chain": nonconvex,
        "learned_warm_start": {
            "heldout_512": {k: lsum[k] for k in ("images", "iters_zero", "iters_warm", "ms_zero",
                                                  "ms_warm", "fallbacks", "all_converged")},
            "headline_image": {"ms_warm": float(np.median(warm_ms)), "iterations_warm": rw[1],
                               "converged": bool(rw[3]), "fallback": bool(rw[4]),
                               "ms_zero": ms_step, "iterations_zero": iters},
            "net_inference_ms_1024": net_ms,
            "net_tflops": net_flop / (net_ms * 1e-3) / 1e12,
            "net_tensor_roofline": {"bound": "tensor", "achieved": net_flop / (net_ms * 1e-3) / 1e12,
                                    "peak": bf16_peak[0], "unit": "TFLOP/s",
                                    "frac": net_flop / (net_ms * 1e-3) / 1e12 / bf16_peak[0],
                                    "peak_kind": bf16_peak[1],
                                    "note": "every layer on tcgen05 (the first from the image "
                                            "rows built by two loader warps, the others fed by TMA "
                                            "in the channel-group layout, the head in the last "
                                            "layer's epilogue), launched with a programmatic "
                                            "dependency; FLOP count of the dense "
                                            "16->32->32->32->16 network, including the zero-padded "
                                            "input channels and the 15 unused output channels"},
            "workload": "held-out seeds 20000.. at 512x512, lambda ~ U[0.05,0.3]; network "
                        "trained on 2000 images (seeds 10000..11999) by the library's kernels",
        },
        "clocks": clk,
    }
    if rank == 0 and world == 1:
        result["cpu_baseline"] = cpu_baseline(f_np, args.cpu_seconds, np.tile(base, (8, 1)), CHAIN_LAM)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
