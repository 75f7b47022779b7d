#!/usr/bin/env python
"""Benchmark of the Wiener-filter MAP hot path on GB300.

Workload (default ``cmb_1024``): the band-power simulation batch of a CMB
temperature patch, 1024 x 1024 pixels of 2 arcmin, analytic C_l, scan-striped
noise, 15% galactic band plus 500 point-source holes; 120 maps = 100 noise-bias
simulations + 20 Fisher simulations, all solved together.  Mixed precision:
FP32 fields and FFTs, FP64 reductions and L-BFGS scalars.

One step = one device L-BFGS iteration (memory 10) on every map of the batch:
the direction from the two-loop recursion, one objective+gradient evaluation
in Hessian-vector form (inverse column stage, row stage, forward column stage,
adjoint), the exact step and the state update.  The metric is objective+gradient
evaluations per second = maps x steps / time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own batch (weak scaling, no collective on
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "objective+grad evals/s"
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=120)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--m", type=int, default=10)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-bandpower", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-solves", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the single-map and 512^2 eval loops, the heterogeneous batch and the ALU peaks")
    ap.add_argument("--fft-variant", type=int, default=0,
                    help="force an FFT-stage variant (wf_opts.fft_variant code); 0 = autotune")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="working precision of the timed iteration (fp64: the plain FP64 path, for its counters)")
    ap.add_argument("--eval-only", action="store_true",
                    help="only the objective+gradient pass (wf_eval) over the batch, for kernel profiles")
    return ap.parse_args()


def config(args, world):
    return {"workload": f"cmb_{args.n}: {args.batch} maps of {args.n}x{args.n} (100 noise-bias + 20 Fisher "
                        f"simulations), 20 log l-bands, "
                        f"{'FP64' if args.precision == 'fp64' else 'mixed FP32/FP64'}",
            "n": args.n, "maps_per_gpu": args.batch, "lbfgs_m": args.m, "precision": args.precision,
            "step": "one L-BFGS iteration on every map (1 Hessian-vector evaluation each)",
            "l2_policy": "working set per step (~20 GB) far exceeds the 126 MB L2; no flush needed",
            "parallelism": f"independent batches per GPU x{world}"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
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
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_problem(args, rank, dev):
    import numpy as np
    import torch
    from paper_1810_00503_gb300 import synth, wf
    inp = synth.cmb_patch(args.n, seed=3)
    B = args.batch
    g = torch.Generator(device=dev)
    g.manual_seed(1000 + rank)
    wdt = torch.float64 if getattr(args, "precision", "mixed") == "fp64" else torch.float32
    Ninv1 = torch.as_tensor(inp.Ninv, dtype=wdt, device=dev)
    Ninv = Ninv1.unsqueeze(0).expand(B, -1, -1, -1).contiguous()
    mask = torch.as_tensor(inp.mask, dtype=torch.uint8, device=dev)
    P = torch.as_tensor(inp.P_half, dtype=wdt, device=dev)
    prob = wf.Problem(torch.zeros_like(Ninv), mask, Ninv, P, precision=getattr(args, "precision", "mixed"),
                      lbfgs_m=args.m)
    z = torch.randn(B, 1, args.n, args.n, generator=g, device=dev, dtype=wdt)
    sig = torch.where(Ninv > 0, torch.rsqrt(torch.clamp(Ninv, min=1e-30)), torch.zeros_like(Ninv))
    noise = torch.randn(B, 1, args.n, args.n, generator=g, device=dev, dtype=wdt) * sig
    d = prob.simulate(z, noise)
    prob.set_data(d)
    torch.cuda.synchronize()
    host = dict(mask=inp.mask, Ninv=inp.Ninv.astype(np.float32), P=inp.P_half.astype(np.float32),
                d=d.float().cpu().numpy())
    return prob, host


def algorithmic_bytes(n, m, elt=4):
    """Compulsory DRAM bytes per map of each kernel of one iteration (ring full).
    Packed vector V = n * n/2 complex = n^2 values; sqrt(P) table n (n/2+1)
    values; weight map n^2 values.
    comb:   reads the 2m stored vectors (the newest pair once: it also carries the
            pending update) and g; writes g and p; reads and writes s once every
            m - 1 launches, when the steps taken since are folded into it (the
            average over that cycle is counted).
    colinv: reads p and sqrt(P).        row: reads W (Hp needs no data map).
    colfwd: reads g, writes q (p is re-read there only because the column
            stages are split; the re-read and the scratch traffic are not counted).
    qdots:  reads q and the m - 1 other stored Q."""
    V = n * n * elt
    sp = n * (n // 2 + 1) * elt
    fold = max(1, m - 1)
    return {"comb": (2 * m + 3) * V + 2 * V / fold, "colinv": V + sp, "row": n * n * elt, "colfwd": 2 * V,
            "qdots": m * V}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_lb_comb_dram_traffic.txt")


def kernel_source_hash():
    """Hash of what decides k_lb_comb's memory traffic: the kernel's own source
    text and the streaming constants it is compiled with."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_1810_00503_gb300/csrc/wf_lbfgs.cuh")).read()
    a = src.index("wf_lb_comb(const WfGeo& g")
    b = src.index("// ----", a)
    consts = open(os.path.join(ROOT, "paper_1810_00503_gb300/csrc/wf_internal.h")).read()
    keep = "\n".join(re.findall(r"#define WF_(?:COMB_\w+|STREAM_GROUP|MAXM)\b.*", consts))
    return hashlib.sha256((src[a:b] + keep).encode()).hexdigest()


def measured_traffic(kernel, maps):
    """DRAM bytes of one launch of `kernel` over `maps` maps, from the committed
    ncu capture (dram__bytes_read.sum + dram__bytes_write.sum per map of a
    smaller batch; the kernel streams every vector once, so traffic scales with
    the maps).  None when no capture exists for this kernel or the kernel's
    source has changed since it was taken."""
    try:
        kv = {}
        for line in open(TRAFFIC_FILE):
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                kv[k] = v
        if kv.get("kernel") != kernel or kv.get("source_sha256") != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_map"]) * maps
    except (OSError, KeyError, ValueError):
        return None


def run_ours(args, rank, world, dev):
    import torch
    from paper_1810_00503_gb300 import wf
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        prob, host = make_problem(args, rank, dev)
        prob.start(gtol_rel=0.0, dchi2_abs=0.0, max_iter=1 << 30, check_every=1, use_graphs=1,
                   refresh_every=0, fft_variant=args.fft_variant)
        prob.step(args.warmup, sync=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = Clocks(torch.cuda.current_device()) if rank == 0 else None
    if clk:
        clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        prob.step(args.steps, sync=False)
        e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop() if clk else None
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    # per-kernel durations of the same iterations, events on the working stream
    with torch.cuda.stream(stream):
        kms = prob.profile(max(3, min(args.steps, 10)))
        active = prob.step(0, sync=True)
        res = prob.finish()
    torch.cuda.synchronize()
    out = dict(ms=ms, kernel_ms=kms, active=active, stats0=res.stats[0], prob=prob, host=host, clocks=clocks)
    return out


def run_e2e(args, dev, host, iters):
    """End to end through the public API from pinned host buffers: copy the
    batch's inputs to the device, prepare, solve `iters` iterations, copy the
    MAP spectra back."""
    import numpy as np
    import torch
    from paper_1810_00503_gb300 import wf
    B, n = args.batch, args.n
    h_d = torch.from_numpy(np.ascontiguousarray(host["d"])).pin_memory()
    h_N = torch.from_numpy(np.ascontiguousarray(host["Ninv"][None].repeat(B, 0))).pin_memory()
    h_m = torch.from_numpy(np.ascontiguousarray(host["mask"])).pin_memory()
    h_P = torch.from_numpy(np.ascontiguousarray(host["P"])).pin_memory()
    h_s = torch.empty((B, 1, n, n // 2 + 1), dtype=torch.complex64).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_d, h_N, h_m, h_P))
    d2h = h_s.numel() * h_s.element_size()
    stream = torch.cuda.Stream(device=dev)
    times, evals = [], []
    for rep in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            d = h_d.to(dev, non_blocking=True)
            N = h_N.to(dev, non_blocking=True)
            msk = h_m.to(dev, non_blocking=True)
            P = h_P.to(dev, non_blocking=True)
            prob = wf.Problem(d, msk, N, P, precision="mixed", lbfgs_m=args.m)
            res = prob.solve(gtol_rel=0.0, max_iter=iters, check_every=iters, use_graphs=1)
            h_s.copy_(res.s, non_blocking=True)
        stream.synchronize()
        dt = time.perf_counter() - t0
        prob.close()
        times.append(dt)
        # one operator pass per map per L-BFGS iteration, as in the device-timed value
        # (the start-up gradient and the final chi^2 pass are not counted)
        evals.append(sum(s["iters"] for s in res.stats))
    dt = min(times)
    ev = evals[times.index(dt)]
    # the same job on a fresh handle: its first solve of the shape times the FFT-stage variants
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        h = wf.Handle()
        prob = wf.Problem(h_d.to(dev, non_blocking=True), h_m.to(dev, non_blocking=True),
                          h_N.to(dev, non_blocking=True), h_P.to(dev, non_blocking=True), precision="mixed",
                          lbfgs_m=args.m, handle=h)
        res = prob.solve(gtol_rel=0.0, max_iter=iters, check_every=iters, use_graphs=1)
        h_s.copy_(res.s, non_blocking=True)
    stream.synchronize()
    cold = time.perf_counter() - t0
    prob.close()
    h.close()
    return {"value": ev / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / iters, "d2h_bytes_per_step": d2h / iters,
            "iterations": iters, "evals": ev, "seconds": dt, "seconds_fresh_handle": cold,
            "note": "one wf_map_solve job from pinned host inputs incl. preparation, on a handle whose FFT-stage "
                    "tuning for this shape is cached (a serving process keeps its handle); seconds_fresh_handle "
                    "is the same job on a new handle, tuning included; bytes per step = job bytes / iterations"}


def run_eval_pass(args, dev, prob, hbm, reps=20, B=None, n=None):
    """The objective + gradient pass itself (wf_eval: steps A1-A5, no L-BFGS)
    over the whole batch, device-timed on its stream.  Algorithmic bytes per
    pass: read s, d and W, write the gradient, and the sqrt(P) table once
    (shared by the maps); the scratch round trips between the three stages are
    not counted."""
    import torch
    B = args.batch if B is None else B
    n = args.n if n is None else n
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    s = torch.randn((B, 1, n, n // 2 + 1), generator=g, device=dev, dtype=prob._cplx())
    grad = torch.empty_like(s)
    chi2 = torch.empty(B, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(3):
            prob.eval(s, grad, chi2, stream=stream)
        e0.record(stream)
        for _ in range(reps):
            prob.eval(s, grad, chi2, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    nh = n * (n // 2 + 1)
    e = 8 if prob._cplx() == torch.complex128 else 4  # bytes of the working type
    alg = B * (2 * e * nh + e * n * n + e * n * n + 2 * e * nh) + e * nh
    achieved = alg / (ms / 1000.0) / 1e9
    # what the three-stage structure must move besides: the packed scratch
    # (n * n/2 complex per map) written by the inverse column stage, read and
    # written by the row stage, read by the forward column stage, and s read a
    # second time by the forward column stage's epilogue
    staged = alg + B * (4 * 2 * e * n * (n // 2) + 2 * e * nh)
    return {"evals_per_s": B * 1000.0 / ms, "ms_per_pass": ms, "maps": B,
            "algorithmic_bytes_per_pass": alg, "achieved_GBps": achieved, "peak_GBps": hbm, "frac": achieved / hbm,
            "staged": {"bytes_per_pass": staged, "GBps": staged / (ms / 1000.0) / 1e9,
                       "frac": staged / (ms / 1000.0) / 1e9 / hbm,
                       "what": "algorithmic bytes plus the scratch round trip between the three stages and the "
                               "epilogue's second read of s (a model of the structure's traffic, not a counter)"},
            "note": "wf_eval on the whole batch (A1-A5: inverse column, row and forward column stages)"}


def run_eval_shapes(args, dev, hbm):
    """The objective + gradient pass on two more workloads: one 1024^2 map
    alone (latency-bound: one map cannot fill the GPU) and 256 maps of 512^2."""
    import types
    out = {}
    for key, n, B, reps in (("single_1024", 1024, 1, 200), ("batch_256x512", 512, 256, 20)):
        prob, _ = make_problem(types.SimpleNamespace(n=n, batch=B, m=args.m), 0, dev)
        out[key] = run_eval_pass(args, dev, prob, hbm, reps=reps, B=B, n=n)
        out[key].pop("note", None)
        prob.close()
    return out


def run_eval_any(dev, hbm, B=64, ny=768, nx=768, reps=10):
    """wf_eval_any (the mixed-radix path for sides that are not powers of two)
    on B maps of ny x nx in mixed precision, device-timed per call on its
    stream; each call includes its scratch allocation, free and stream
    synchronisation.  Algorithmic bytes: read s, d, the mask (1 byte a pixel)
    and Ninv, write the gradient, and P once (shared by the maps)."""
    import torch
    from paper_1810_00503_gb300 import wf
    g = torch.Generator(device=dev)
    g.manual_seed(6)
    h1 = nx // 2 + 1
    s = torch.randn((B, 1, ny, h1), generator=g, device=dev, dtype=torch.complex64)
    d = torch.randn((B, 1, ny, nx), generator=g, device=dev)
    mask = (torch.rand((B, ny, nx), generator=g, device=dev) > 0.2).to(torch.uint8)
    Ninv = torch.rand((B, 1, ny, nx), generator=g, device=dev) + 0.5
    P = torch.rand((1, ny, h1), generator=g, device=dev)
    grad = torch.empty_like(s)
    chi2 = torch.empty(B, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        for _ in range(3):
            wf.eval_any(s, mask, Ninv, P, d=d, chi2=chi2, grad=grad, stream=stream)
        e0.record(stream)
        for _ in range(reps):
            wf.eval_any(s, mask, Ninv, P, d=d, chi2=chi2, grad=grad, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    e, N, nh = 4, ny * nx, ny * h1
    alg = B * (2 * e * nh + e * N + N + e * N + 2 * e * nh) + e * nh
    achieved = alg / (ms / 1000.0) / 1e9
    return {"evals_per_s": B * 1000.0 / ms, "ms_per_call": ms, "maps": B, "shape": [ny, nx],
            "algorithmic_bytes_per_call": alg, "achieved_GBps": achieved, "frac": achieved / hbm,
            "note": "wf_eval_any, mixed precision, radix 4 x 4 x 4 x 4 x 3 transforms; per call including its "
                    "scratch allocation, free and synchronisation"}


def run_hetero(args, dev, count=256, n_bands=10, sizes=(64, 128, 256, 512, 1024)):
    """Heterogeneous batch: `count` independent maps of n in {64, 128, 256,
    512, 1024} (uneven masks, noise levels and spectral slopes), one problem
    per size, all solved as one batch by wf_map_solve_many (each iteration one
    set of seven launches shared by every size, one CUDA graph per round) to
    ||g|| / ||g0|| < 1e-6 in mixed precision;
    then d chi^2 / d log q for n_bands log-spaced bands at the solutions
    through the adjoint stage (wf_eval_bands)."""
    import numpy as np
    import torch
    from paper_1810_00503_gb300 import synth, wf
    maps = synth.hetero_batch(count=count, seed=4, sizes=sizes)
    groups = {}
    for mp in maps:
        groups.setdefault(mp.n, []).append(mp)
    probs, sizes = [], []
    for n in sorted(groups):
        ms = groups[n]
        B = len(ms)
        f32 = lambda a: torch.as_tensor(np.stack(a), dtype=torch.float32, device=dev).contiguous()
        Ninv = f32([mp.Ninv for mp in ms])
        mask = torch.as_tensor(np.stack([mp.mask for mp in ms]), dtype=torch.uint8, device=dev)
        P = f32([mp.P_half for mp in ms])
        prob = wf.Problem(torch.zeros_like(Ninv), mask, Ninv, P, precision="mixed", lbfgs_m=args.m)
        prob.set_data(prob.simulate(f32([mp.z for mp in ms]), f32([mp.noise for mp in ms])))
        probs.append(prob)
        sizes.append((n, B))
    torch.cuda.synchronize()
    wf.solve_many(probs, gtol_rel=1e-6, max_iter=2)  # tunes each size's tiles, sets up the solvers
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = wf.solve_many(probs, gtol_rel=1e-6, max_iter=20000, check_every=32, refresh_every=200)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    evals = sum(st["evals"] for r in res for st in r.stats)
    per = {str(n): {"maps": B, "iterations_mean": float(np.mean([st["iters"] for st in r.stats])),
                    "fft_variant": p.variant()} for (n, B), r, p in zip(sizes, res, probs)}
    statuses = sorted({st["status"] for r in res for st in r.stats})
    # d chi^2 / d log q at the solutions
    bands = [torch.as_tensor(wf.band_table(n, np.geomspace(1.0, n / 2, n_bands + 1)), device=dev)
             for n, _ in sizes]
    reps = 10
    for p, r, bt in zip(probs, res, bands):
        p.eval_bands(r.s, bt, n_bands)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        for p, r, bt in zip(probs, res, bands):
            p.eval_bands(r.s, bt, n_bands)
    torch.cuda.synchronize()
    dq_dt = (time.perf_counter() - t0) / reps
    for p in probs:
        p.close()
    return {"maps": count, "sizes": per, "seconds": dt, "map_solves_per_s": count / dt,
            "evals_per_s": evals / dt, "stop": "||g||/||g0|| < 1e-6", "statuses": statuses,
            "dchi2_dlogq": {"bands": n_bands, "ms_per_batch": dq_dt * 1e3, "maps_per_s": count / dq_dt},
            "note": "one problem per size, all sizes solved as one batch by wf_map_solve_many: each iteration "
                    "is seven launches shared by the five sizes (ping-pong stages, tile widths tuned per size), each "
                    "round of 32 iterations one graph launch; a 2-iteration solve first tunes and sets up the solvers"}


def run_alu_peaks():
    """Measured FMA throughput (wf_alu_peak), TFLOP/s."""
    from paper_1810_00503_gb300 import wf
    return {"fp32_tflops": wf.alu_peak("f32") / 1e12, "fp64_tflops": wf.alu_peak("f64") / 1e12,
            "how": "independent FMA chains on every SM's resident blocks, about 40 ms each"}


def run_map_solves(args, dev, n=512, maps=120):
    """MAP solves/s: `maps` simulated CMB maps of n^2 solved together to the
    paper's stopping rule (Delta chi^2 < 0.1), mixed precision."""
    import torch
    from paper_1810_00503_gb300 import synth, wf
    inp = synth.cmb_patch(n, seed=3)
    g = torch.Generator(device=dev)
    g.manual_seed(91)
    Ninv = torch.as_tensor(inp.Ninv, dtype=torch.float32, device=dev)
    mask = torch.as_tensor(inp.mask, dtype=torch.uint8, device=dev)
    P = torch.as_tensor(inp.P_half, dtype=torch.float32, device=dev)
    sig = torch.where(Ninv > 0, torch.rsqrt(torch.clamp(Ninv, min=1e-30)), torch.zeros_like(Ninv))
    Nb = Ninv[None].expand(maps, 1, n, n).contiguous()
    prob = wf.Problem(torch.zeros_like(Nb), mask, Nb, P, precision="mixed", lbfgs_m=args.m)
    d = prob.simulate(torch.randn(maps, 1, n, n, generator=g, device=dev),
                      torch.randn(maps, 1, n, n, generator=g, device=dev) * sig)
    prob.set_data(d)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = prob.solve(gtol_rel=0.0, dchi2_abs=0.1, max_iter=20000, check_every=32, refresh_every=200)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    its = [st["iters"] for st in res.stats]
    prob.close()
    return {"map_solves_per_s": maps / dt, "seconds": dt, "n": n, "maps": maps, "stop": "Delta chi^2 < 0.1",
            "iterations_mean": float(sum(its) / len(its)), "iterations_max": max(its),
            "statuses": sorted({st["status"] for st in res.stats})}


def run_bandpower(args, dev, n_sim=100, n_bands=20, n_fd=1):
    """One complete band-power estimate (Sec. 2.4-2.5) on the same CMB patch:
    n_sim noise-bias simulations and n_bands * n_fd Fisher simulations, all
    solved with the paper's stopping rule (Delta chi^2 < 0.1), on the device."""
    import numpy as np
    import torch
    from paper_1810_00503_gb300 import synth, wf
    n = args.n
    inp = synth.cmb_patch(n, seed=3)
    g = torch.Generator(device=dev)
    g.manual_seed(77)
    Ninv = torch.as_tensor(inp.Ninv, dtype=torch.float32, device=dev)
    mask = torch.as_tensor(inp.mask, dtype=torch.uint8, device=dev)
    P = torch.as_tensor(inp.P_half, dtype=torch.float32, device=dev)
    sig = torch.where(Ninv > 0, torch.rsqrt(torch.clamp(Ninv, min=1e-30)), torch.zeros_like(Ninv))
    one = wf.Problem(torch.zeros_like(Ninv)[None], mask, Ninv[None], P, precision="mixed")
    d = one.simulate(torch.randn(1, 1, n, n, generator=g, device=dev),
                     torch.randn(1, 1, n, n, generator=g, device=dev) * sig)[0]
    one.close()
    bands = torch.as_tensor(np.ascontiguousarray(synth.log_bands(n, n_bands)[..., : n // 2 + 1]), dtype=torch.int16,
                            device=dev)
    z = torch.randn(n_sim, 1, n, n, generator=g, device=dev)
    nz = torch.randn(n_sim, 1, n, n, generator=g, device=dev) * sig
    u = torch.randn(n_bands, n_fd, 1, n, n, generator=g, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, stats = wf.bandpower_estimate(d, mask, Ninv, P, bands, n_bands, z, nz, u, precision="mixed",
                                       gtol_rel=0.0, dchi2_abs=0.1, max_iter=20000, check_every=32,
                                       refresh_every=200)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nsim = n_sim + n_bands * n_fd
    its = [st["iters"] for st in stats]
    return {"sims_per_s": nsim / dt, "map_solves_per_s": (nsim + 1) / dt, "seconds": dt,
            "n_sim": n_sim, "n_fisher": n_bands * n_fd, "n_bands": n_bands, "stop": "Delta chi^2 < 0.1",
            "iterations_mean": float(np.mean(its)), "iterations_max": int(np.max(its)),
            "statuses": sorted(set(st["status"] for st in stats)),
            "theta_hat_over_fid_median": float(np.median(res["theta_hat"] / res["theta_fid"]))}


def run_eb_bandpower(args, dev, n=512, n_bands=8, n_sim=20, n_fd=2):
    """Joint E/B band powers (App. C) on the 512^2 shear workload, n_bands E and
    n_bands B bands: the full Fisher form (a Fisher map per band and Fisher
    simulation) and the leakage-bias form (per-band maps for the E bands, one
    joint B map per Fisher simulation), same fields and stopping rule as the
    CMB estimate."""
    import numpy as np
    import torch
    from paper_1810_00503_gb300 import synth, wf
    inp = synth.shear_eb(n, seed=2)
    g = torch.Generator(device=dev)
    g.manual_seed(78)
    Ninv = torch.as_tensor(inp.Ninv, dtype=torch.float32, device=dev)
    mask = torch.as_tensor(inp.mask, dtype=torch.uint8, device=dev)
    P = torch.as_tensor(inp.P_half, dtype=torch.float32, device=dev)
    sig = torch.where(Ninv > 0, torch.rsqrt(torch.clamp(Ninv, min=1e-30)), torch.zeros_like(Ninv))
    one = wf.Problem(torch.zeros_like(Ninv)[None], mask, Ninv[None], P, precision="mixed")
    d = one.simulate(torch.randn(1, 2, n, n, generator=g, device=dev),
                     torch.randn(1, 2, n, n, generator=g, device=dev) * sig)[0]
    one.close()
    nbt = 2 * n_bands
    bands = torch.as_tensor(np.ascontiguousarray(synth.log_bands(n, n_bands, C=2)[..., : n // 2 + 1]),
                            dtype=torch.int16, device=dev)
    z = torch.randn(n_sim, 2, n, n, generator=g, device=dev)
    nz = torch.randn(n_sim, 2, n, n, generator=g, device=dev) * sig
    uE = torch.randn(n_bands, n_fd, 2, n, n, generator=g, device=dev)
    uB = torch.randn(n_bands, n_fd, 2, n, n, generator=g, device=dev)
    forms = {"full": (torch.cat([uE, uB]), 0), "leakage_bias": (torch.cat([uE, uB[:1]]), n_bands)}
    out = {"workload": f"shear_eb {n}^2, {n_bands} E + {n_bands} B bands, {n_sim} noise-bias simulations, "
                       f"{n_fd} Fisher simulations per Fisher row, mixed FP32/FP64, stop Delta chi^2 < 0.1"}
    for name, (u, split) in forms.items():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, stats = wf.bandpower_estimate(d, mask, Ninv, P, bands, nbt, z, nz, u, precision="mixed",
                                           gtol_rel=0.0, dchi2_abs=0.1, max_iter=20000, check_every=32,
                                           refresh_every=200, leak_split=split)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        its = [st["iters"] for st in stats]
        out[name] = {"seconds": dt, "estimates_per_s": 1.0 / dt, "map_solves": len(stats),
                     "map_solves_per_s": len(stats) / dt, "iterations_mean": float(np.mean(its)),
                     "statuses": sorted(set(st["status"] for st in stats)),
                     "theta_hat_over_fid_median_E": float(np.median(res["theta_hat"][:n_bands]
                                                                    / res["theta_fid"][:n_bands]))}
    out["leakage_bias_speedup"] = out["full"]["seconds"] / out["leakage_bias"]["seconds"]
    return out


FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64


# FP64 FLOPs of one L-BFGS iteration counted by ncu on the FP64 path (DFMA as
# two; profiles/fp64_iteration_cmb1024_counters.md), per (n, m).
FP64_ITERATION_FLOPS_COUNTED = {(1024, 10): 158.3e6}


def iteration_flops(n, m):
    """FP64 arithmetic of one L-BFGS iteration on one n x n map (C = 1): the
    ncu-counted figure where there is one, else a model (5 L log2 L per
    complex FFT of length L: two real 2-D transforms; 5m + 9 complex dot
    products or real-coefficient axpys per packed value, 4 flops each; about
    10 flops per value for the per-mode and per-pixel steps), which
    overcounts the radix-8/16 butterflies.  Returns (flops, source)."""
    import math
    if (n, m) in FP64_ITERATION_FLOPS_COUNTED:
        return FP64_ITERATION_FLOPS_COUNTED[(n, m)], "ncu FP64 instruction counters"
    h = n // 2
    fft = 5 * (h * n * math.log2(n) + n * h * math.log2(h))
    vals = n * h
    return 2 * fft + vals * (4 * (5 * m + 9) + 10), "model"


def run_fp64_reference(args, dev, cert_tol=1e-4, fp64_peak=None):
    """Certified accuracy, mixed against the plain single-map FP64 GPU path, on
    map 0 of the workload.  Both solve the same map (FP32-rounded inputs) with
    wf_map_solve_refined to the error certificate |grad chi2| / 2 <= cert_tol |s|
    (a bound on the relative L2 error of the MAP, since the whitened
    half-Hessian has every eigenvalue >= 1): the mixed path with FP32 operator
    passes and FP64 outer residuals, the FP64 path in FP64 throughout.  Also the
    FP64 path's iteration throughput against the measured FP64 FMA peak."""
    import torch
    from paper_1810_00503_gb300 import synth, wf
    n = args.n
    inp = synth.cmb_patch(n, seed=3)
    g = torch.Generator(device=dev)
    g.manual_seed(1000)
    Ninv64 = torch.as_tensor(inp.Ninv, dtype=torch.float64, device=dev)
    mask = torch.as_tensor(inp.mask, dtype=torch.uint8, device=dev)
    P64 = torch.as_tensor(inp.P_half, dtype=torch.float64, device=dev)
    sig = torch.where(Ninv64 > 0, torch.rsqrt(torch.clamp(Ninv64, min=1e-30)), torch.zeros_like(Ninv64))
    z = torch.randn(1, 1, n, n, generator=g, device=dev, dtype=torch.float64)
    nz = torch.randn(1, 1, n, n, generator=g, device=dev, dtype=torch.float64) * sig
    p64 = wf.Problem(torch.zeros_like(Ninv64)[None], mask, Ninv64[None], P64, precision="fp64", lbfgs_m=args.m)
    d64 = p64.simulate(z, nz)
    d32, N32, P32 = d64.float(), Ninv64.float()[None], P64.float()
    p64.close()
    p64 = wf.Problem(d32.double(), mask, N32.double(), P32.double(), precision="fp64", lbfgs_m=args.m)
    p32 = wf.Problem(d32, mask, N32, P32, precision="mixed", lbfgs_m=args.m)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        p64.start(gtol_rel=0.0, max_iter=1 << 30, check_every=1)
        p64.step(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p64.step(args.steps, sync=False)
        e1.record(stream)
        torch.cuda.synchronize()
        it_ms = e0.elapsed_time(e1) / args.steps
        p64.finish()
    torch.cuda.synchronize()
    out = {}
    opts = dict(cert_tol=cert_tol, max_rounds=8, gtol_rel=1e-5, max_iter=50000, check_every=64)
    for name, p in (("mixed", p32), ("fp64", p64)):
        p.solve_refined(**opts)  # first solve of the shape: the FFT-stage tuning
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r, c = p.solve_refined(**opts)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "certificate": float(c[0]), "iterations": r.stats[0]["iters"],
                     "status": r.stats[0]["status"]}
    p64.close()
    p32.close()
    flops, flops_src = iteration_flops(n, args.m)
    achieved = flops / (it_ms / 1000.0) / 1e12
    peak = fp64_peak or FP64_PEAK_TFLOPS
    src = ("measured on this GPU (wf_alu_peak, FP64 FMA chains)" if fp64_peak
           else "nominal GB300 FP64 rate (no measured FP64 peak)")
    return {"certified": {"tol": cert_tol, "mixed": out["mixed"], "fp64": out["fp64"],
                          "mixed_speedup": out["fp64"]["seconds"] / out["mixed"]["seconds"],
                          "how": "wf_map_solve_refined on map 0 of the workload, first round to |g|/|g0| < 1e-5"},
            "fp64_single_map_evals_per_s": 1000.0 / it_ms, "fp64_single_map_ms_per_iteration": it_ms,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "flops_per_iteration": flops, "flops_source": flops_src,
                         "peak_source": src}}


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_sample(args, budget_s=12.0, host=None):
    """Textbook FP64 L-BFGS (the oracle) on one map of the same workload,
    as many iterations as fit in about budget_s seconds; returns evals/s."""
    import numpy as np
    from oracle import wf_oracle as O
    from paper_1810_00503_gb300 import synth
    inp = synth.cmb_patch(args.n, seed=3)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    W = inp.mask[None] * inp.Ninv
    count = [0]
    t_end = [None]

    def fg(z):
        count[0] += 1
        r = d - O.apply_A(z, inp.P)
        return float(np.sum(z * z) + np.sum(r * W * r)), 2.0 * (z - O.apply_At(W * r, inp.P))

    state = {"t0": None}

    def cb(it, x, f, g):
        if time.perf_counter() - state["t0"] > budget_s:
            raise StopIteration

    fg(np.zeros_like(d))  # warm-up of numpy's FFT plans
    count[0] = 0
    state["t0"] = time.perf_counter()
    try:
        O.lbfgs(fg, np.zeros_like(d), m=args.m, gtol_rel=0.0, max_iter=10 ** 6, callback=cb)
    except StopIteration:
        pass
    dt = time.perf_counter() - state["t0"]
    return count[0] / dt, count[0], dt


def cores_used():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    """The oracle as the reference arm: K steps of its textbook L-BFGS on one
    1024^2 map of the same workload (bounded sample), on the host cores."""
    import numpy as np
    from oracle import wf_oracle as O
    from paper_1810_00503_gb300 import synth
    inp = synth.cmb_patch(args.n, seed=3)
    d = O.synthesize_data(inp.z, inp.noise, inp.mask, inp.P)
    W = inp.mask[None] * inp.Ninv
    count = [0]

    def fg(z):
        count[0] += 1
        r = d - O.apply_A(z, inp.P)
        return float(np.sum(z * z) + np.sum(r * W * r)), 2.0 * (z - O.apply_At(W * r, inp.P))

    marks = []

    def cb(it, x, f, g):
        marks.append((time.perf_counter(), count[0]))
        if it >= args.warmup + args.steps:
            raise StopIteration

    try:
        O.lbfgs(fg, np.zeros_like(d), m=args.m, gtol_rel=0.0, max_iter=args.warmup + args.steps, callback=cb)
    except StopIteration:
        pass
    (t0, c0), (t1, c1) = marks[args.warmup - 1], marks[-1]
    dt = t1 - t0
    steps = len(marks) - args.warmup
    value = (c1 - c0) / dt
    cores = 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, 1),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"one {args.n}^2 map of the batch, {steps} textbook L-BFGS iterations "
                                       f"(numpy FP64, single-threaded pocketfft)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    from paper_1810_00503_gb300 import build, wf
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)
    if not os.path.exists(wf.LIB_PATH):
        if rank == 0:
            build.build()
        if world > 1:
            torch.distributed.barrier()
    if args.eval_only:
        prob, _ = make_problem(args, rank, dev)
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
        print(json.dumps({"eval_pass": run_eval_pass(args, dev, prob, hbm, reps=args.steps)}), flush=True)
        prob.close()
        return
    r = run_ours(args, rank, world, dev)
    B, K = args.batch, args.steps
    value = world * B * K / (r["ms"] / 1000.0)
    ab = algorithmic_bytes(args.n, args.m)
    names = ["comb", "colinv", "row", "colfwd", "qdots", "scalar"]
    kms = dict(zip(names, r["kernel_ms"]))
    dom = max(names[:5], key=lambda k: kms[k])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    achieved = ab[dom] * B / (kms[dom] / 1000.0) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": r["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic", "config": config(args, world),
            "gpu_launches": 6 * K,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": measured_traffic(dom, B), "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": ab[dom] * B,
                         "kernel_ms": kms,
                         "iteration_frac": sum(ab[k] for k in names[:5]) * B
                         / (sum(kms.values()) / 1000.0) / 1e9 / hbm},
            "solver": {"maps_active_after": r["active"], "chi2_map0": r["stats0"]["chi2"],
                       "gnorm_rel_map0": r["stats0"]["gnorm_rel"],
                       "fft_variant": r["prob"].variant(),
                       "fft_variant_source": "forced" if args.fft_variant else "autotuned"}}
    if rank == 0:
        line["clocks"] = r["clocks"]
        line["eval_pass"] = run_eval_pass(args, dev, r["prob"], hbm)
        ep = line["eval_pass"]
        line["roofline"]["eval_pass"] = {"what": "wf_eval objective+gradient pass over the batch (3 FFT stages)",
                                         "achieved": ep["achieved_GBps"], "frac": ep["frac"],
                                         "ms": ep["ms_per_pass"], "algorithmic_bytes": ep["algorithmic_bytes_per_pass"],
                                         "staged_frac": ep["staged"]["frac"]}
        r["prob"].close()
        if not args.no_extra:
            line["eval_shapes"] = run_eval_shapes(args, dev, hbm)
            line["eval_shapes"]["any_64x768"] = run_eval_any(dev, hbm)
        if not args.no_solves:
            line["map_solves"] = run_map_solves(args, dev)
        if not args.no_extra:
            line["hetero"] = run_hetero(args, dev)
        alu = run_alu_peaks() if not args.no_extra else {}
        if alu:
            line["alu_peaks"] = alu
        if not args.no_bandpower:
            line["bandpower"] = run_bandpower(args, dev)
            try:
                line["eb_bandpower"] = run_eb_bandpower(args, dev)
            except Exception as e:  # a side measurement: report it, keep the line
                line["eb_bandpower"] = {"error": f"{type(e).__name__}: {e}"}
        if not args.no_e2e:
            line["e2e"] = run_e2e(args, dev, r["host"], iters=max(K, 10))
        if not args.no_cpu:
            v, cnt, dt = oracle_sample(args)
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"textbook FP64 L-BFGS on one {args.n}^2 map of the batch, "
                                              f"{cnt} objective+gradient evaluations in {dt:.1f} s "
                                              f"(single-threaded numpy), of {cores_used()} host cores"}
        if not args.no_fp64:  # last in the line: the certified mixed-against-FP64 comparison
            line["fp64_reference"] = run_fp64_reference(args, dev, fp64_peak=alu.get("fp64_tflops"))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
