"""Benchmark of the GB300 TV-L1 optical-flow library.

Workload (default): one 640 x 480 pair -- gradient-noise texture under an affine motion (rotation
2 deg, zoom 1.03, translation (3, -2)) plus a 120 x 80 box moving (6, 4), noise sigma 0.01 --
solved with pADMM (c = 0.05, a = 8, beta = 0.05, lambda = 5) over 5 pyramid levels (scale 0.5),
10 warps per level and 100 inner iterations per warp: 409.2 Mpix*iter per flow.  A step is one
whole solve of that pair (every row of the hot path: pyramid, level transfer, derivatives,
warping, inner iterations, residual/energy reductions).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 (torchrun, one rank per GPU) every rank solves its own copy of the workload
(independent pairs: weak scaling, no data-path collective); value = pairs of all ranks / max
rank time.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "flows/s & Mpix·iter/s vs plain GPU at EPE≤1e-2px to FP64; p50/p99 latency"
H, W = 480, 640
LEVELS, WARPS, ITERS = 5, 10, 100
LAM, BETA = 5.0, 0.05
WORKLOAD = "640x480 affine+box pair, pADMM, 5 levels x 10 warps x 100 iters"


def mpix_iter_per_flow(levels=LEVELS, warps=WARPS, iters=ITERS, h=H, w=W, eta=0.5, lo=0):
    import math
    hs, ws = [h], [w]
    for _ in range(1, levels):
        hs.append(max(1, int(math.floor(hs[-1] * eta + 0.5))))
        ws.append(max(1, int(math.floor(ws[-1] * eta + 0.5))))
    return sum(hs[l] * ws[l] for l in range(lo, levels)) * warps * iters / 1e6


def reduce_max_over_ranks(values, device=None):
    """Max over all ranks of each timing value (a no-op on one rank).  Works with any
    torch.distributed backend (NCCL on the GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(units_per_rank, n_ranks, t_max):
    """Weak scaling: every rank processes `units_per_rank` independent pairs; the job's rate is
    all ranks' units over the slowest rank's time."""
    return units_per_rank * n_ranks / t_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9 for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_oracle_solves(threads, out_level=0):
    """Times the FP64 oracle, as it stands, on the bench pair's schedule down to `out_level`:
    `threads` host threads each solve their own copy of the pair at once (the oracle's C code
    releases the GIL, so they run in parallel on the host cores).  Returns (Mpix*iter/s, wall
    seconds, Mpix*iter per solve, the first solve's flow)."""
    import concurrent.futures as cf
    import oracle
    from paper_2011_10979_gb300 import synth
    oracle.build()
    pr = synth.affine_rect_pair()
    P = oracle.Params(method=0, lam=LAM, beta=BETA, levels=LEVELS, warps=WARPS, iters=ITERS, out_level=out_level)
    with cf.ThreadPoolExecutor(threads) as ex:
        t = time.perf_counter()
        futs = [ex.submit(oracle.solve, pr.I0, pr.I1, P) for _ in range(threads)]
        res = [f.result() for f in futs]
        dt = time.perf_counter() - t
    work = mpix_iter_per_flow(lo=out_level)
    return work * threads / dt, dt, work, res[0][:2]


def run_reference(args):
    """The reference arm: there is no reference implementation, only the paper, so this times the
    FP64 oracle on the host cores.  A step is one bounded sample of the bench workload: every host
    thread solves levels 1..4 of the 640x480 schedule (102.0 of its 409.2 Mpix*iter per flow;
    the finest level is left out to keep the run within minutes).  The throughput unit is the
    bench's flows/s, counting a sample as 102.0 / 409.2 of a flow."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    threads = host_threads()
    per_flow = mpix_iter_per_flow()
    times, rates = [], []
    for k in range(args.warmup + args.steps):
        rate, dt, work, _ = cpu_oracle_solves(threads, out_level=1)
        if k >= args.warmup:
            times.append(dt)
            rates.append(rate)
    t_step = float(np.mean(times))
    units = threads * work / per_flow          # flows per step
    value = units / t_step
    desc = ("levels 1..4 of the 640x480 schedule (%.1f of %.1f Mpix*iter per flow), one solve per thread on %d "
            "threads per step; a sample counts as %.3f flow" % (work, per_flow, threads, work / per_flow))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "flows/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc, "units_per_step": units},
            "mpix_iter_per_s": float(np.mean(rates)),
            "cpu_baseline": {"value": value, "unit": "flows/s", "cores": threads, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "flows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batch16(args):
    """The batch leg alone on 16 uneven pairs (BF16 duals + FP32 flow, strip heights autotuned
    unless --rows-per-warp sets one), one timed batch: a short command for profiling the batched
    kernels.  Streaming engine on every
    level, as in the 256-pair batch, where no level has few enough small pairs for the
    level-resident launch."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2011_10979_gb300 import flow
    from paper_2011_10979_gb300.build import build
    build()
    r = batch_measure(flow, torch, dev, n=16, fp32_flow=1, steps=1, engine=flow.OF_ENGINE_STREAM,
                      rows_per_warp=args.rows_per_warp)
    print(json.dumps({"legs": "batch16", "batch": r}))


def run_level(args):
    """Single-level solves for a profiler: the 40x30 and 640x480 levels of the bench pair's kind
    (one warp, 30 inner iterations, three solves each) of --method (pADMM unless set) on the given
    engine, strip height --rows-per-warp (ADMM only; unset: the built-in rule, which on the
    streaming engine runs these levels three iterations per launch on the tile kernel, as ALG1
    does).  A pinned height runs the row-streaming kernel, whose 40x30 level shows the latency of
    one warp's row steps; with --method pdr the 640x480 level runs the one-launch pDR tile kernel."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2011_10979_gb300 import flow, synth
    from paper_2011_10979_gb300.build import build
    build()
    ctx = flow.Context(0)
    eng = {"stream": flow.OF_ENGINE_STREAM, "persistent": flow.OF_ENGINE_PERSISTENT, "fused": flow.OF_ENGINE_FUSED}
    ty = args.rows_per_warp if args.rows_per_warp > 0 else 0
    for (h, w) in ((30, 40), (480, 640)):
        pr = synth.affine_rect_pair(h, w) if h >= 120 else synth.random_affine_rect_pair(h, w, 3)
        I0, I1 = torch.from_numpy(pr.I0).to(dev), torch.from_numpy(pr.I1).to(dev)
        method = {"padmm": flow.OF_PADMM_I, "pdr": flow.OF_PDR, "alg1": flow.OF_CP}[args.method]
        P = flow.default_params(lam=LAM, beta=BETA, levels=1, warps=1, iters=30, engine=eng[args.engine],
                                method=method, rows_per_warp=ty if method == flow.OF_PADMM_I else 0)
        for _ in range(3):
            flow.of_solve(ctx, I0, I1, P, stats=False)
        torch.cuda.synchronize(dev)
    ctx.close()
    print(json.dumps({"legs": "level", "method": args.method, "engine": args.engine, "rows_per_warp": ty}))


def run_serving(args):
    """The serving leg alone, at its sustained and its overload rate for 60 s each (one GPU)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2011_10979_gb300 import flow
    from paper_2011_10979_gb300.build import build
    build()
    out = {rate: serving_measure(flow, torch, dev, rate_hz=rate, duration_s=60.0, drain_s=10.0)
           for rate in (50.0, 200.0)}
    print(json.dumps({"legs": "serving", "serving_60s": {"%.0f_req_per_s" % k: v for k, v in out.items()}}))


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2011_10979_gb300 import flow, synth
    from paper_2011_10979_gb300.build import build
    build()
    ctx = flow.Context(dev.index)
    pr = synth.affine_rect_pair(seed=1 + rank)
    I0, I1 = torch.from_numpy(pr.I0).to(dev), torch.from_numpy(pr.I1).to(dev)
    P = flow.default_params(method=flow.OF_PADMM_I, lam=LAM, beta=BETA, levels=LEVELS, warps=WARPS, iters=ITERS)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2

    def step():
        return flow.of_solve(ctx, I0, I1, P, stats=False)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(dev.index)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    sampler.start()
    for k in range(args.steps):
        flush.zero_()                       # evict the previous step's data from L2
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    barrier()
    clocks = sampler.stop()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_step = float(np.sum(ms)) / args.steps / 1e3
    # end to end through the host entry point: pinned host images in, host flow out
    h0 = torch.from_numpy(pr.I0).pin_memory()
    h1 = torch.from_numpy(pr.I1).pin_memory()
    hu = torch.empty((H, W), dtype=torch.float32).pin_memory()
    hv = torch.empty((H, W), dtype=torch.float32).pin_memory()
    for _ in range(2):
        flow.of_solve_host_ptrs(ctx, h0.data_ptr(), h1.data_ptr(), H, W, P, hu.data_ptr(), hv.data_ptr())
    barrier()
    t0 = time.perf_counter()
    n_e2e = max(3, args.steps)
    for _ in range(n_e2e):
        flow.of_solve_host_ptrs(ctx, h0.data_ptr(), h1.data_ptr(), H, W, P, hu.data_ptr(), hv.data_ptr())
    barrier()
    t_e2e = (time.perf_counter() - t0) / n_e2e
    t_step, t_e2e = reduce_max_over_ranks([t_step, t_e2e], dev)
    # dominant kernel: the streaming pADMM iteration at the finest level, timed inside the solve graph
    launches = flow.of_solve_kernel_count(ctx, H, W, P)
    full = args.legs == "all"
    roof = kernel_roofline(flow, torch, dev, pr) if full else None
    t_plain = serving = serving50 = batch = batch_all16 = batch_fp32 = prec_line = solvers = None
    if full:
        # plain single-pair FP32 GPU path (one kernel per operator), same workload
        Pp = flow.default_params(method=flow.OF_PADMM_I, lam=LAM, beta=BETA, levels=LEVELS, warps=WARPS, iters=ITERS,
                                 engine=flow.OF_ENGINE_PLAIN)
        flow.of_solve(ctx, I0, I1, Pp, stats=False)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            flow.of_solve(ctx, I0, I1, Pp, stats=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t_plain = e0.elapsed_time(e1) / 3 / 1e3
        serving = serving_measure(flow, torch, dev, rate_hz=50.0)
        serving50 = serving_measure(flow, torch, dev, rate_hz=200.0)
        batch = batch_measure(flow, torch, dev, fp32_flow=1)
        batch_all16 = batch_measure(flow, torch, dev, fp32_flow=0)
        batch_fp32 = batch_measure(flow, torch, dev, prec=flow.OF_PREC_FP32)
        prec_line = precision_measure(flow, torch, dev)
        solvers = solvers_measure(flow, torch, dev, I0, I1, pr)
    if rank != 0:
        return
    cpu = None
    if ws == 1 and full:
        # the whole schedule, no extrapolation: one solve on one thread, then one per host thread
        r1, dt1, work, (ou, ov) = cpu_oracle_solves(1)
        threads = host_threads()
        rn, dtn, _, _ = cpu_oracle_solves(threads)
        # accuracy of the timed GPU path against the oracle on the bench pair itself
        gu, gv, _, _ = flow.of_solve(ctx, I0, I1, P, stats=False)
        gu, gv = gu.double().cpu().numpy(), gv.double().cpu().numpy()
        cpu = {"value": rn / work, "unit": "flows/s", "cores": threads, "kind": "oracle",
               "sample": "the whole 640x480 schedule (%.1f Mpix*iter), one solve per thread on %d threads at once, "
                         "%.1f s" % (work, threads, dtn),
               "single_thread": {"value": r1 / work, "unit": "flows/s", "seconds": dt1},
               "epe_vs_gpu_px": float(np.hypot(gu - ou, gv - ov).mean()),
               "max_abs_du_px": float(np.max(np.abs(gu - ou))), "max_abs_dv_px": float(np.max(np.abs(gv - ov)))}
    work = mpix_iter_per_flow()
    value = whole_job_rate(1, ws, t_step)
    line = {"metric": METRIC, "value": value, "unit": "flows/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H, "W": W, "levels": LEVELS, "warps": WARPS, "iters": ITERS,
                       "method": "pADMM", "lambda": LAM, "beta": BETA, "storage": "fp32",
                       "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if ws > 1 else "single"},
            "mpix_iter_per_s": work * ws / t_step,
            "plain_gpu": {"value": 1.0 / t_plain, "unit": "flows/s", "engine": "plain (one kernel per operator)",
                          "speedup": t_plain / t_step} if full else None,
            "roofline": roof,
            "batch": batch,
            "serving": serving,
            "serving_overload_200hz": serving50,
            "batch_all16": batch_all16,
            "batch_fp32": batch_fp32,
            "precision_1024x436": prec_line,
            "solvers_640x480": solvers,
            "cpu_baseline": cpu,
            "e2e": {"value": whole_job_rate(1, ws, t_e2e), "unit": "flows/s", "h2d_bytes_per_step": 2 * H * W * 4,
                    "d2h_bytes_per_step": 2 * H * W * 4},
            "gpu_launches": int(launches) * args.steps,
            "clocks": clocks}
    if not full:
        line["legs"] = args.legs
    print(json.dumps(line), flush=True)


_BATCH_PAIRS = {}


def batch_pairs(n):
    """The n distinct seeded pairs of the uneven-size batch, rendered once per process on the host
    threads (spawned workers; input generation only)."""
    if n not in _BATCH_PAIRS:
        from paper_2011_10979_gb300 import synth
        ranks = max(1, int(os.environ.get("LOCAL_WORLD_SIZE", os.environ.get("WORLD_SIZE", "1"))))
        _BATCH_PAIRS[n] = synth.batch_pairs(n=n, workers=max(1, min(16, (os.cpu_count() or 1) // ranks)))
    return _BATCH_PAIRS[n]


def batch_measure(flow, torch, dev, n=256, prec=None, fp32_flow=1, steps=2, engine=None, rows_per_warp=-1):
    """Uneven-size batch: n distinct pairs, each with its own seed, sizes drawn uniformly from
    {96x64, 320x240, 640x480, 1024x436, 1242x375}, affine+box motion up to 15 px, BF16 storage,
    FP32 last warp, 5 levels x 10 warps x 100 iterations, solved with of_solve_batch (one
    work-list launch per inner iteration for all pairs).  The streaming kernel's strip height is
    autotuned per level on the (untimed) first solve unless rows_per_warp sets it."""
    prec = flow.OF_PREC_BF16 if prec is None else prec
    pairs = batch_pairs(n)
    I0 = [torch.from_numpy(p.I0).to(dev) for p in pairs]
    I1 = [torch.from_numpy(p.I1).to(dev) for p in pairs]
    P = flow.default_params(method=flow.OF_PADMM_I, lam=LAM, beta=BETA, levels=LEVELS, warps=WARPS, iters=ITERS,
                            precision=prec, fp32_last_warp=1, fp32_flow=fp32_flow, rows_per_warp=rows_per_warp,
                            engine=flow.OF_ENGINE_FUSED if engine is None else engine)
    flow.of_solve_batch(flow_ctx_batch(flow, dev), I0, I1, P, stats=False)
    torch.cuda.synchronize(dev)
    rows = flow.of_rows_per_warp(flow_ctx_batch(flow, dev), [p.I0.shape for p in pairs], P)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        flow.of_solve_batch(flow_ctx_batch(flow, dev), I0, I1, P, stats=False)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t = e0.elapsed_time(e1) / steps / 1e3
    work = sum(mpix_iter_per_flow(h=p.I0.shape[0], w=p.I0.shape[1]) for p in pairs)   # Mpix*iter
    bpp = 92.0 if prec == flow.OF_PREC_FP32 else (58.0 if fp32_flow else 46.0)
    name = {0: "fp32", 1: "fp16", 2: "bf16"}[prec] + ("" if prec == flow.OF_PREC_FP32 else
                                                        ("_duals+fp32_flow" if fp32_flow else "_all"))
    return {"workload": "%d distinct seeded pairs of uneven sizes, pADMM, 5x10x100" % n,
            "storage": name, "value": n / t, "unit": "flows/s",
            "rows_per_warp": {"mode": "autotuned" if P.rows_per_warp == -1 else "set", "per_level": rows},
            "s_per_batch": t, "gpix_iter_per_s": work / 1e3 / t,
            "effective_gbs": work * 1e6 * bpp / t / 1e9, "bytes_per_px_iter": bpp}


_BATCH_CTX = {}


def flow_ctx_batch(flow, dev):
    if dev.index not in _BATCH_CTX:
        _BATCH_CTX[dev.index] = flow.Context(dev.index)
    return _BATCH_CTX[dev.index]


def precision_measure(flow, torch, dev):
    """The 1024 x 436 layered pair (6 levels x 10 warps x 150 iterations) with FP32, FP16 and BF16
    storage (FP32 last warp): device time per solve and the EPE of the 16-bit results against
    the FP32 result."""
    from paper_2011_10979_gb300 import synth
    pr = synth.layered_pair()
    I0, I1 = torch.from_numpy(pr.I0).to(dev), torch.from_numpy(pr.I1).to(dev)
    ctx = flow_ctx_batch(flow, dev)
    out, ref = {}, None
    for prec, ff, name in ((flow.OF_PREC_FP32, 1, "fp32"), (flow.OF_PREC_FP16, 1, "fp16_duals+fp32_flow"),
                           (flow.OF_PREC_BF16, 1, "bf16_duals+fp32_flow"), (flow.OF_PREC_FP16, 0, "fp16_all"),
                           (flow.OF_PREC_BF16, 0, "bf16_all")):
        P = flow.default_params(lam=LAM, beta=BETA, levels=6, warps=10, iters=150, precision=prec, fp32_last_warp=1,
                                fp32_flow=ff)
        u, v, _, _ = flow.of_solve(ctx, I0, I1, P, stats=False)
        torch.cuda.synchronize(dev)
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            u, v, _, _ = flow.of_solve(ctx, I0, I1, P, stats=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 3
        if ref is None:
            ref = (u.clone(), v.clone())
        epe = float(torch.hypot(u - ref[0], v - ref[1]).mean())
        out[name] = {"ms_per_solve": ms, "flows_per_s": 1e3 / ms, "epe_vs_fp32_px": epe,
                     "max_abs_du_vs_fp32_px": float((u - ref[0]).abs().max())}
    return out


def solvers_measure(flow, torch, dev, I0, I1, pr):
    """Every solver of the library on the bench workload (640 x 480, 5 levels x 10 warps x 100
    iterations, FP32, default engines), as the paper's Sec. 4 compares them: device time per
    solve and the end-point error against the pair's known motion (where it is defined)."""
    ctx = flow.Context(dev.index or 0)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for name, kw in (("pADMM", dict(method=flow.OF_PADMM_I, r=1.0)), ("rpADMMI", dict(method=flow.OF_PADMM_I, r=1.618)),
                     ("rpADMMII", dict(method=flow.OF_PADMM_II, rho=1.9)),
                     ("Zach-pADMM", dict(method=flow.OF_PADMM_I, r=1.0, beta=0.0)),
                     ("pDR", dict(method=flow.OF_PDR)), ("ALG1", dict(method=flow.OF_CP))):
        kw = dict(dict(lam=LAM, beta=BETA, levels=LEVELS, warps=WARPS, iters=ITERS), **kw)
        P = flow.default_params(**kw)
        u, v, _, _ = flow.of_solve(ctx, I0, I1, P, stats=False)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            u, v, _, _ = flow.of_solve(ctx, I0, I1, P, stats=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 3
        r = {"ms_per_solve": ms, "flows_per_s": 1e3 / ms, "launches": flow.of_solve_kernel_count(ctx, H, W, P)}
        if pr.u_true is not None:
            ut = torch.from_numpy(pr.u_true.astype(np.float32)).to(dev)
            vt = torch.from_numpy(pr.v_true.astype(np.float32)).to(dev)
            r["epe_vs_true_px"] = float(torch.hypot(u - ut, v - vt).mean())
        out[name] = r
    # the per-pixel s-preconditioner (a~_ij = M_s(ij)) against the scalar a~ = max M_s, with the
    # stopping rule on (tol 1e-3): iterations run, time and accuracy
    for mode, name in ((0, "pADMM tol=1e-3, scalar a~"), (1, "pADMM tol=1e-3, per-pixel a~")):
        P = flow.default_params(lam=LAM, beta=BETA, levels=LEVELS, warps=WARPS, iters=ITERS, tol=1e-3,
                                a_tilde_mode=mode)
        u, v, _, st = flow.of_solve(ctx, I0, I1, P)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            flow.of_solve(ctx, I0, I1, P, stats=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / 3
        r = {"ms_per_solve": ms, "flows_per_s": 1e3 / ms, "iters_run": st["iters_run"], "energy": st["energy"]}
        if pr.u_true is not None:
            ut = torch.from_numpy(pr.u_true.astype(np.float32)).to(dev)
            vt = torch.from_numpy(pr.v_true.astype(np.float32)).to(dev)
            r["epe_vs_true_px"] = float(torch.hypot(u - ut, v - vt).mean())
        out[name] = r
    ctx.close()
    return out


SERVE_DIST = ("Poisson arrivals, sizes {320x240: 40%, 640x480: 30%, 1024x436: 20%, 1920x1080: 8%, 3840x2160: 2%}, "
              "layered motion <= 30 px, BF16 duals + FP32 flow, 5 levels x 10 warps x 100 iterations")


def serving_measure(flow, torch, dev, rate_hz=50.0, duration_s=15.0, drain_s=5.0, max_active=32):
    """The serving loop under Poisson arrivals (rate_hz for duration_s) of the serving size mix
    (one seeded layered pair per size, reused).  Every step of the loop advances all admitted
    requests by one warp, their inner iterations sharing launches.  Throughput counts the requests
    finished inside the arrival window; after it the loop gets drain_s to finish the rest, and
    what is still queued or running then is reported as unfinished (past saturation the queue only
    grows).  Latency = submit to result on the host, p50/p99 over the finished requests.  Beside it,
    the same request sequence through one of_solve call at a time (the plain single-pair path):
    the sum of the per-size device times of a solve."""
    from paper_2011_10979_gb300 import synth
    imgs = {}
    for (H, W), _ in synth.SERVE_MIX:
        imgs[(H, W)] = synth.layered_pair(H, W, seed=40 + H, max_shift=30.0, sigma=0.01)
    arrivals = synth.poisson_arrivals(rate_hz, duration_s, seed=5)
    sizes = synth.serve_sizes(len(arrivals), seed=4)
    P = flow.default_params(method=flow.OF_PADMM_I, lam=LAM, beta=BETA, levels=LEVELS, warps=WARPS, iters=ITERS,
                            precision=flow.OF_PREC_BF16, fp32_last_warp=1, fp32_flow=1)
    ctx = flow.Context(dev.index)
    # the plain single-pair path: device time of one whole solve per size
    stream = torch.cuda.current_stream(dev)
    single_ms = {}
    for k, pr in imgs.items():
        I0, I1 = torch.from_numpy(pr.I0).to(dev), torch.from_numpy(pr.I1).to(dev)
        flow.of_solve(ctx, I0, I1, P, stats=False)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            flow.of_solve(ctx, I0, I1, P, stats=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        single_ms[k] = e0.elapsed_time(e1) / 2
    flow.of_server_start(ctx, P, 0, max_active)
    try:
        warm = [(flow.of_server_submit(ctx, imgs[k].I0, imgs[k].I1), k) for k in imgs]  # pinned pool, memory pool
        for rid, k in warm:
            while flow.of_server_poll(ctx, rid, k) is None:
                time.sleep(0.001)
        pending, lat, done_at, lat_size = {}, [], [], {}
        t0 = time.perf_counter()
        nxt = 0
        while (nxt < len(arrivals) or pending) and time.perf_counter() - t0 < duration_s + drain_s:
            now = time.perf_counter() - t0
            while nxt < len(arrivals) and arrivals[nxt] <= now:
                k = sizes[nxt]
                pending[flow.of_server_submit(ctx, imgs[k].I0, imgs[k].I1)] = k
                nxt += 1
            for rid in list(pending):
                r = flow.of_server_poll(ctx, rid, pending[rid])
                if r is not None:
                    lat.append(r[2])
                    lat_size.setdefault(pending[rid], []).append(r[2])
                    done_at.append(time.perf_counter() - t0)
                    del pending[rid]
            time.sleep(0.0005)
        unfinished = len(pending) + (len(arrivals) - nxt)
    finally:
        flow.of_server_stop(ctx)
        ctx.close()
    lat = np.array(lat)
    in_window = int(np.sum(np.array(done_at) <= duration_s))
    work = sum(mpix_iter_per_flow(h=h, w=w) for h, w in sizes[:len(lat)])
    seq_s = sum(single_ms[k] for k in sizes) / 1e3
    return {"workload": "%s, %.0f req/s for %.0f s" % (SERVE_DIST, rate_hz, duration_s),
            "offered": len(arrivals), "finished": int(len(lat)), "finished_in_window": in_window,
            "unfinished_after_drain": int(unfinished), "drain_s": drain_s,
            "value": in_window / duration_s, "unit": "flows/s",
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "gpix_iter_per_s": work / 1e3 / (done_at[-1] if done_at else 1.0), "max_active": max_active,
            "p50_p99_ms_by_size": {"%dx%d" % (w, h): [round(float(np.percentile(v, 50)), 1),
                                                      round(float(np.percentile(v, 99)), 1), len(v)]
                                   for (h, w), v in sorted(lat_size.items())},
            "single_pair_path": {"value": len(sizes) / seq_s, "unit": "flows/s",
                                 "note": "the same requests through one of_solve at a time (device time)",
                                 "ms_per_solve": {"%dx%d" % (w, h): round(v, 3) for (h, w), v in single_ms.items()}}}


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the pADMM kernel that runs the
# 640 x 480 level of the bench solve (ncu, cold cache): k_admm_tile2, three iterations per launch,
# 16.00 MB read (the 13 input planes once), 0 written (the written planes stay in L2).  Set to None
# whenever that kernel changes, until it is captured again.
TILE2_640_DRAM_BYTES = 16.00e6
ITERS_PER_LAUNCH = 3


def kernel_roofline(flow, torch, dev, pr, reps=20):
    """Per-launch time of the pADMM kernel on the 640 x 480 level where it runs: inside the solve's
    CUDA graph.  With the bench's fixed schedule that level runs three inner iterations per launch
    (k_admm_tile2).  Two graph-launched single-level solves of the bench pair, with 220 and 20 inner
    iterations, are timed with CUDA events on their stream; the difference / 200 is one iteration
    (with its share of graph launch gaps), three of them one launch.  Algorithmic traffic: 13
    planes read + 10 written, FP32 = 92 B per pixel-iteration, 276 B per pixel and launch."""
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    ctx = flow.Context(dev.index or 0)
    I0 = torch.from_numpy(pr.I0.astype(np.float32)).to(dev)
    I1 = torch.from_numpy(pr.I1.astype(np.float32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    t = {}
    for iters in (20, 220):
        P = flow.default_params(lam=LAM, beta=BETA, levels=1, warps=1, iters=iters, engine=flow.OF_ENGINE_STREAM)
        for _ in range(3):
            flow.of_solve(ctx, I0, I1, P, stats=False)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            flow.of_solve(ctx, I0, I1, P, stats=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t[iters] = e0.elapsed_time(e1) / reps / 1e3
    ctx.close()
    per = (t[220] - t[20]) / 200.0 * ITERS_PER_LAUNCH   # one launch = three iterations
    bytes_per_launch = ITERS_PER_LAUNCH * 92.0 * H * W
    achieved = bytes_per_launch / per / 1e9
    # the level's working set stays in L2: its bandwidth for a working set of the same size
    # (half read, half written, streamed 400 times in one launch)
    l2 = flow.of_l2_bandwidth(int(bytes_per_launch / ITERS_PER_LAUNCH), 400)
    return {"kernel": "k_admm_tile2<float,float,1,0,32> (640x480 level, three iterations per launch)",
            "bound": "hbm", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": src,
            "traffic": TILE2_640_DRAM_BYTES, "us_per_launch": per * 1e6,
            "us_per_iteration": per * 1e6 / ITERS_PER_LAUNCH, "algorithmic_bytes_per_launch": bytes_per_launch,
            "timing": "graph-launched single-level solves, (t(220 iters) - t(20 iters)) / 200 x 3 per launch",
            "l2_peak": l2, "frac_of_l2": achieved / l2,
            "note": "the 640x480 level's 28 MB state stays in the 129 MB L2 between iterations; l2_peak is the "
                    "library's L2 streaming probe over a 28 MB read+write working set"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    # "solve": only the timed single-pair solve (and its e2e leg), e.g. as a short command to run
    # under a profiler; "batch16": only a 16-pair batch (one GPU), likewise; "all" (default) adds the
    # roofline, plain, batch, serving, precision, solver and CPU-baseline legs
    ap.add_argument("--legs", default="all", choices=["all", "solve", "batch16", "serving", "level"])
    # the level leg: single-level solves for a profiler (engine and strip height as given)
    ap.add_argument("--engine", default="stream", choices=["stream", "persistent", "fused"])
    ap.add_argument("--method", default="padmm", choices=["padmm", "pdr", "alg1"])
    # strip height of the batch16 leg (-1: autotuned; a fixed height makes the launch sequence
    # independent of timing, e.g. under a profiler)
    ap.add_argument("--rows-per-warp", type=int, default=-1, choices=[-1, 0, 1, 2, 8, 32])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.legs == "batch16":
        run_batch16(args)
    elif args.legs == "serving":
        run_serving(args)
    elif args.legs == "level":
        run_level(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
