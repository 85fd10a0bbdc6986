#!/usr/bin/env python
"""Benchmark: walker-steps/s of the multideterminant hot path (Psi, grad Psi/Psi,
Lap Psi/Psi and E_L for every walker) on the chlorine-like 750k-determinant
workload, one JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision mixed|fp64]

A step evaluates the whole batch of walkers (8,192 per GPU) once. Walkers are
independent, so with N GPUs each rank evaluates its own 8,192 walkers (weak
scaling, no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/s (Ψ,∇Ψ,∇²Ψ), 17e⁻, N_det=750k: mixed vs FP64 at 1e-5 rel err"
UNIT = "walker-steps/s"
CPU_SAMPLE_WALKERS = 96     # bounded oracle sample for the CPU baseline (~10-30 s of CPU work)
CPU_SINGLE_CORE_WALKERS = 8  # the same oracle on one core, for the per-core figure
# dram__bytes_read.sum + dram__bytes_write.sum of the average k_spmm_seg launch on the 750k workload
# with 8,192 walkers, from one ncu capture of the current kernel per (precision, walker chunks):
# mixed in three chunks of 6, 21 and 5 tiles (the six launches of one evaluation), FP64 in one; null
# for a configuration that was not captured
SPMM_TRAFFIC_750K = {("mixed", 3): 182.7e6, ("fp64", 1): 602.1e6}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    parts = [p for p in vis.split(",") if p.strip()]
    if local_rank < len(parts) and parts[local_rank].strip().isdigit():
        return int(parts[local_rank])
    return local_rank


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.strip().lower().startswith("model name"):
                return l.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for l in open("/proc/cpuinfo"):
            if l.lower().startswith(("model name", "cpu model")):
                return l.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline(wl, n_sample, threads=None, single_core=CPU_SINGLE_CORE_WALKERS):
    """The FP64 oracle as it stands, on a bounded sample of walkers, all host
    cores; then on one core for a smaller sample (the per-core figure, the unit
    the paper's timings use)."""
    import oracle
    threads = threads or os.cpu_count() or 1
    R = wl.R[:n_sample]
    t0 = time.perf_counter()
    ref = oracle.evaluate(wl, R=R, n_threads=threads)
    dt = time.perf_counter() - t0
    cb = {"value": n_sample / dt, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu_model": cpu_model(),
          "sample": "%d of the %d walkers of one step (same expansion), %.1f s wall" % (n_sample, wl.n_walk, dt)}
    if single_core:
        t0 = time.perf_counter()
        oracle.evaluate(wl, R=wl.R[:single_core], n_threads=1)
        d1 = time.perf_counter() - t0
        cb["single_core"] = {"value": single_core / d1, "unit": UNIT, "cores": 1,
                             "ms_per_walker_step": d1 * 1e3 / single_core,
                             "sample": "%d walkers on one thread, %.1f s" % (single_core, d1)}
    return ref, cb


def fp64_peak(device, clock_index=None):
    """The FP64 FMA pipe's throughput, measured now on this device by the
    library's probe (independent FMA chains on every SM), with the SM clocks seen
    while it ran."""
    import paper_1510_00730_gb300 as pkg
    pkg.measure_fp64_rate(device, fma_per_thread=1 << 16, reps=2)  # warm the clocks
    with ClockSampler(clock_index if clock_index is not None else device) as clk:
        tf, ms, mhz = pkg.measure_fp64_rate(device, fma_per_thread=1 << 19, reps=12)
    summ = clk.summary()
    summ["in_kernel_sm_mhz"] = mhz
    return tf, ms, summ


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same workload and metric."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    from paper_1510_00730_gb300 import synth
    wl = synth.WORKLOADS[args.workload]()
    n = max(1, min(args.ref_sample, wl.n_walk))
    for _ in range(args.warmup):
        cpu_baseline(wl, max(1, n // 4))
    times = []
    cores = os.cpu_count() or 1
    for s in range(args.steps):
        lo = (s * n) % max(1, wl.n_walk - n)
        t0 = time.perf_counter()
        import oracle
        oracle.evaluate(wl, R=wl.R[lo:lo + n], n_threads=cores)
        times.append(time.perf_counter() - t0)
    per = statistics.mean(times)
    val = n / per
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "walkers_per_gpu": wl.n_walk, "n_det": int(wl.n_det),
                       "n_elec": wl.n_elec, "sampled_walkers_per_step": n},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d walkers per step of the %d-walker workload" % (n, wl.n_walk)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PROFILED_STEPS = 3  # untimed steps with the library's stage events, after the timed ones


def _time_steps(ctx, Rdev, out, flush, stream, steps, warmup, dist, clock_index=None):
    """Warm up, then time `steps` evaluations with CUDA events (L2 flushed between
    steps outside the events, the library's own stage events off). Then a few more
    steps with the stage events on, for the per-stage times and the timeline of the
    last one. Returns per-step ms, per-stage ms, clocks and that timeline."""
    import torch
    for s in range(warmup):
        ctx.evaluate(Rdev[s % len(Rdev)], out=out)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(clock_index) if clock_index is not None else None
    if clk:
        clk.__enter__()
    ctx.set_profiling(2)  # the contraction kernels' own global-timer stamps: no events in the streams
    contract_ms = []
    for s in range(steps):
        flush.fill_(float(s))          # evict L2 between timed steps (outside the events)
        torch.cuda.synchronize()       # the step starts on an idle device
        ev[s][0].record(stream)
        ctx.evaluate(Rdev[s % len(Rdev)], out=out)
        ev[s][1].record(stream)
        contract_ms.append(ctx.profile()["contract"])  # waits for this step's contraction events
    torch.cuda.synchronize()
    if clk:
        clk.__exit__(None, None, None)
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ctx.set_profiling(True)
    stage_ms, prof_ms = [], []
    for s in range(PROFILED_STEPS):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        ctx.evaluate(Rdev[s % len(Rdev)], out=out)
        stage_ms.append(ctx.profile())  # waits for this step's events
        prof_ms.append(ctx.timeline()["end"])
    timeline = ctx.timeline()
    timeline["profiled_step_ms"] = statistics.median(prof_ms)
    ctx.set_profiling(False)
    kern = {k: statistics.median(d[k] for d in stage_ms) for k in stage_ms[0]}
    kern["contract_timed"] = statistics.mean(contract_ms)
    return step_ms, kern, (clk.summary() if clk else None), timeline


def rank_batches(wl, rank, n_batches=4):
    """Walker batches of one rank: distinct per rank (seeded by the rank), the
    workload's own walkers as rank 0's first batch."""
    import numpy as np

    from paper_1510_00730_gb300 import synth
    rng = np.random.default_rng(1000 + rank)
    return [wl.R if (b == 0 and rank == 0) else synth.make_walkers(rng, wl.n_walk, wl.n_elec)
            for b in range(n_batches)]


def whole_job_value(walkers_per_rank, world, ms):
    """Walker-steps/s of the whole job: every rank's walkers over the max-over-ranks step time."""
    return walkers_per_rank * world / (ms / 1e3)


def _max_over_ranks(x, dist, dev):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args):
    import numpy as np
    import torch

    import paper_1510_00730_gb300 as pkg
    from paper_1510_00730_gb300 import synth

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    world = max(world, 1)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    prec_of = {"mixed": pkg.PRECISION_MIXED, "fp64": pkg.PRECISION_FP64}
    primary = args.precision
    others = [p for p in ("mixed", "fp64") if p != primary] if args.compare else []

    wl = synth.WORKLOADS[args.workload]()
    W = wl.n_walk
    N = wl.n_elec
    # distinct walker batches per rank, resident in HBM before timing
    batches = rank_batches(wl, rank)
    Rdev = [torch.from_numpy(np.ascontiguousarray(b)).to(dev) for b in batches]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    results = {}
    ctxs = {}

    def timed(name, ctx, clock_index=None):
        out = ctx.alloc_outputs(W)
        step_ms, kern, clocks, timeline = _time_steps(ctx, Rdev, out, flush, stream, args.steps, args.warmup,
                                                      dist, clock_index)
        n_fb = int(((out["status"] & pkg.WS_FALLBACK) != 0).sum().item())
        ms = _max_over_ranks(statistics.mean(step_ms), dist, dev)
        n_esc = int(((out["status"] & pkg.WS_ESCALATED) != 0).sum().item())
        results[name] = dict(ms=ms, value=whole_job_value(W, world, ms), kern=kern, clocks=clocks, n_fb=n_fb,
                             n_esc=n_esc, chunks=ctx.last_chunks, kernels=ctx.last_kernels,
                             fallback_tol=ctx.fallback[0], timeline=timeline)

    for pname in [primary] + others:
        ctx = pkg.Context.from_workload(wl, device=local, precision=prec_of[pname])
        if args.fallback_tol is not None and pname == primary:
            ctx.set_fallback(args.fallback_tol)
        if args.chunks is not None:
            ctx.set_walker_chunks(args.chunks)
        ctxs[pname] = ctx
        if pname == primary:
            timed(pname, ctx, _gpu_index(local))
            continue
        # the other precision at the primary's accuracy target (the metric compares the two paths
        # at the same relative error), then at its own default target
        own_tol, own_cap = ctx.fallback
        ctx.set_fallback(ctxs[primary].fallback[0], own_cap)
        timed(pname, ctx)
        ctx.set_fallback(own_tol, own_cap)
        timed(pname + "_default_fallback", ctx)
    # the mixed path with its optional double-float contraction (outside the FP64 contraction of the
    # method's precision plan; reported beside the headline, never as it)
    df_contract = None
    if primary == "mixed" and args.compare:
        c = ctxs["mixed"]
        c.set_tuning(contract_impl=1)
        out = c.alloc_outputs(W)
        step_ms, kern, _, _ = _time_steps(c, Rdev, out, flush, stream, args.steps, args.warmup, dist)
        ms = _max_over_ranks(statistics.mean(step_ms), dist, dev)
        df_contract = dict(value=whole_job_value(W, world, ms), ms_per_step=ms, kernels_ms=kern)
        c.set_tuning(contract_impl=0)
        del out
    st = ctxs[primary].stats()
    main = results[primary]
    main_chunks = main["chunks"]
    # kernels per evaluation, as the library counts them (chunks and fallback included)
    st_launches = main["kernels"]

    # end to end through the host-memory C-ABI call: H2D of R and D2H of all outputs per step
    ctx = ctxs[primary]
    hR = torch.empty((W, N, 3), dtype=torch.float64, pin_memory=True)
    hR.numpy()[:] = batches[0]
    hout = dict(log_abs_psi=torch.empty(W, dtype=torch.float64, pin_memory=True).numpy(),
                sign=torch.empty(W, dtype=torch.int8, pin_memory=True).numpy(),
                grad=torch.empty((W, N, 3), dtype=torch.float64, pin_memory=True).numpy(),
                lap=torch.empty((W, N), dtype=torch.float64, pin_memory=True).numpy(),
                e_local=torch.empty(W, dtype=torch.float64, pin_memory=True).numpy(),
                status=torch.empty(W, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32))
    for _ in range(2):
        ctx.evaluate_host(hR.numpy(), out=hout)
    e2e_t = []
    for s in range(args.steps):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.evaluate_host(hR.numpy(), out=hout)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = _max_over_ranks(statistics.mean(e2e_t) * 1e3, dist, dev)
    h2d = W * N * 3 * 8
    d2h = W * (8 + 1 + 3 * N * 8 + N * 8 + 8 + 4)

    # roofline of the dominant kernel: the FP64 sparse contraction k_spmm_seg, 2 launches per
    # step and walker chunk (v = C r_dn, u = C^T r_up), each 2 FLOP per nonzero per walker;
    # the average launch covers W / chunks walkers
    kern = main["kern"]
    flops_launch = 2.0 * st["n_det"] * W / main_chunks
    launch_ms = kern["contract_timed"] / (2 * main_chunks)
    achieved = flops_launch / (launch_ms / 1e3) / 1e12
    traffic = args.traffic
    if traffic is None and args.workload == "chlorine_like_750k" and W == 8192:
        traffic = SPMM_TRAFFIC_750K.get((primary, main_chunks))
    peak, peak_ms, peak_clocks = fp64_peak(local, _gpu_index(local))
    roofline = {"kernel": "k_spmm_seg", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_source": "measured in this run: FP64 FMA probe (mdet_measure_fp64_rate, 8 independent "
                               "accumulators per thread fed from L1-resident tables, 16 warps per SM, fastest of "
                               "12 launches of %.1f ms)" % peak_ms,
                "peak_clocks": peak_clocks, "peak_nominal": 1.25,
                "flops_per_launch": flops_launch, "launch_ms": launch_ms,
                "launch_ms_source": "mean over the timed steps of each launch's device duration, from its first "
                                    "block's start to its last warp's exit on the GPU global timer (written by the "
                                    "kernel; CUDA events in the pipelined streams lengthen the step by about 10 %)"}

    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if primary == "fp64" else "f64+f32x2",
            "data": "synthetic",
            "config": {"workload": args.workload, "precision": primary, "walkers_per_gpu": W,
                       "n_det": st["n_det"], "n_det_up": st["n_det_up"], "n_det_dn": st["n_det_dn"],
                       "n_elec": N, "n_ao": st["n_ao"], "n_mo": st["n_mo"],
                       "l2": "flushed between timed steps (512 MB write outside the events)",
                       "walker_chunks": main_chunks, "parallelism": "dp%d (walkers)" % world},
            "clocks": main["clocks"],
            "e2e": {"value": whole_job_value(W, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": st_launches * args.steps,
            "kernels_ms": kern,
            "kernels_ms_note": "stage times (library CUDA events, summed over walker chunks) from %d profiled steps "
                               "after the timed ones, whose events lengthen the step (timeline_ms); the timed steps "
                               "record no event: contract_timed sums the contraction kernels' own timer stamps "
                               "(the roofline's launch time)" % PROFILED_STEPS,
            "timeline_ms": {"chunks": [{k: [round(v[0], 3), round(v[1], 3)] for k, v in c.items()}
                                       for c in main["timeline"]["chunks"]],
                            "refine": [round(x, 3) for x in main["timeline"]["refine"]],
                            "end": round(main["timeline"]["end"], 3),
                            "profiled_step_ms_median": round(main["timeline"]["profiled_step_ms"], 3)},
            "fallback_walkers": main["n_fb"], "escalated_walkers": main["n_esc"],
            "roofline": roofline}
    if df_contract is not None:
        line["mixed_df_contraction"] = df_contract
    line["fallback_tol"] = main["fallback_tol"]
    for pname in others:
        for name in (pname, pname + "_default_fallback"):
            line[name] = {"value": results[name]["value"], "ms_per_step": results[name]["ms"],
                          "kernels_ms": results[name]["kern"], "fallback_walkers": results[name]["n_fb"],
                          "fallback_tol": results[name]["fallback_tol"]}

    if rank == 0 and world == 1 and args.batch and args.workload == "chlorine_like_750k":
        # config 4 beside the headline: 64 uneven expansions, autotuned, one graph launch per step
        b = measure_batched(primary, args.steps, args.warmup, args.streams, args.tune_ms)
        line["batched_uneven_64"] = {k: b[k] for k in ("value", "unit", "ms_per_step", "sum_of_solo_ms", "batch_gain",
                                                       "clocks", "gpu_launches", "tuning_histogram")}
        line["batched_uneven_64"].update(b["config"])
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from tests.parity import walker_quantiles
        ref, cb = cpu_baseline(wl, CPU_SAMPLE_WALKERS)
        line["cpu_baseline"] = cb
        acc = {}
        for pname, c in ctxs.items():
            host = c.evaluate_host(batches[0][:CPU_SAMPLE_WALKERS])
            acc[pname] = walker_quantiles(host, ref)
        line["accuracy_vs_oracle"] = dict(walkers=CPU_SAMPLE_WALKERS, **acc)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def measure_batched(precision, steps, warmup, streams=8, tune_ms=60.0, fallback_tol=None):
    """The 64-expansion uneven workload: every expansion autotuned, then all
    evaluations replayed as one CUDA-graph launch; value = walkers of all
    expansions per second of graph time. Returns the JSON line (a dict)."""
    import numpy as np
    import torch

    import paper_1510_00730_gb300 as pkg
    from paper_1510_00730_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    prec = {"mixed": pkg.PRECISION_MIXED, "fp64": pkg.PRECISION_FP64}[precision]
    wls = synth.batched_uneven()
    ctxs = [pkg.Context.from_workload(wl, device=dev.index, precision=prec) for wl in wls]
    if fallback_tol is not None:
        for c in ctxs:
            c.set_fallback(fallback_tol)
    Rs = [torch.from_numpy(wl.R).to(dev) for wl in wls]
    t0 = time.perf_counter()
    tunes = [c.autotune(R, budget_ms=tune_ms) for c, R in zip(ctxs, Rs)]
    tune_s = time.perf_counter() - t0
    batch = pkg.Batch(ctxs, Rs, n_streams=streams)
    batched_kernels = sum(c.last_kernels for c in ctxs)  # as enqueued by the batch (its warm-up pass)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        batch.launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with ClockSampler(_gpu_index(dev.index)) as clk:
        for s in range(steps):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            ev[s][0].record(stream)
            batch.launch()
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    W = sum(wl.n_walk for wl in wls)
    # time of each expansion alone (no batching), for the gain of sharing the GPU, and the roofline
    # of its FP64 contraction (4 FLOP per product and walker; launch times from the kernels' own
    # timer stamps, profiling mode 2, which adds no event to the streams)
    solo = 0.0
    contract_tf = []
    for c, R, wl in zip(ctxs, Rs, wls):
        out = c.alloc_outputs(R.shape[0])
        c.evaluate(R, out=out)
        c.set_profiling(2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        c.evaluate(R, out=out)
        b.record(stream)
        torch.cuda.synchronize()
        solo += a.elapsed_time(b)
        cms = c.profile()["contract"]
        c.set_profiling(False)
        contract_tf.append((4.0 * wl.n_det * wl.n_walk / (cms * 1e-3) / 1e12 if cms > 0 else float("nan"),
                            4.0 * wl.n_det * wl.n_walk, cms))
    peak, _, _ = fp64_peak(dev.index, _gpu_index(dev.index))
    tf = np.array([t[0] for t in contract_tf])
    flops = np.array([t[1] for t in contract_tf])
    weighted = float(flops.sum() / (sum(t[2] for t in contract_tf) * 1e-3) / 1e12)
    line = {"metric": "walker-steps/s, 64 uneven expansions in one graph launch", "value": W / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "higher_is_better": True, "dtype": "f64" if prec == pkg.PRECISION_FP64 else "f64+f32x2",
            "data": "synthetic",
            "config": {"workload": "batched_uneven_64", "precision": precision, "walkers_total": W,
                       "n_det_total": int(sum(wl.n_det for wl in wls)), "streams": streams,
                       "fallback_tol": ctxs[0].fallback[0],
                       "autotune_s": tune_s, "l2": "flushed between timed steps"},
            "sum_of_solo_ms": solo, "batch_gain": solo / ms,
            "roofline_per_expansion": {
                "kernel": "k_spmm_seg", "bound": "alu", "unit": "TFLOP/s", "peak": peak,
                "peak_source": "measured FP64 FMA probe (mdet_measure_fp64_rate), this run",
                "achieved": {"min": float(np.nanmin(tf)), "median": float(np.nanmedian(tf)),
                             "max": float(np.nanmax(tf)), "all_expansions": weighted},
                "frac_median": float(np.nanmedian(tf)) / peak, "frac_all_expansions": weighted / peak,
                "note": "each expansion evaluated alone; all_expansions = total contraction FLOPs over total "
                        "contraction time"},
            "tuning_histogram": {k: dict(zip(*np.unique([t[k] for t in tunes], return_counts=True)))
                                 for k in ("spmm_chunk", "mo_ec", "walker_chunks")},
            "clocks": clk.summary(),
            # kernels per expansion as the library counts them (the solo runs above are not in a
            # batch, so the count of a batched evaluation is taken with the batch's choices)
            "gpu_launches": batched_kernels * steps}
    line["tuning_histogram"] = {k: {str(a): int(b) for a, b in v.items()} for k, v in line["tuning_histogram"].items()}
    batch.close()
    for c in ctxs:
        c.close()
    return line


def run_batched(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(measure_batched(args.precision, args.steps, args.warmup, args.streams, args.tune_ms,
                                     args.fallback_tol)), flush=True)


def run_truncation(args):
    """Synthetic analogue of the paper's truncation table (Table 5) on the
    750k-determinant expansion: for each threshold eps, norm-based truncation
    (Sec. 3, eps_up = eps_dn = eps) against truncation by |c_k| that keeps the
    same number of distinct spin determinants (the paper's measure of cost).
    For each: products kept, distinct determinants, the retained share of
    sum c^2 and walker-steps/s of one evaluation of 8,192 walkers (CUDA
    events, L2 flushed between steps)."""
    import numpy as np
    import torch

    import paper_1510_00730_gb300 as pkg
    from paper_1510_00730_gb300 import synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prec = {"mixed": pkg.PRECISION_MIXED, "fp64": pkg.PRECISION_FP64}[args.precision]
    wl = synth.chlorine_like_750k()
    R = torch.from_numpy(wl.R).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    total = float(np.sum(wl.ci_coef ** 2))

    def timed(mask):
        sub = synth.subset_products(wl, mask)
        ctx = pkg.Context.from_workload(sub, device=0, precision=prec)
        out = ctx.alloc_outputs(wl.n_walk)
        for _ in range(args.warmup):
            ctx.evaluate(R, out=out)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for s in range(args.steps):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            ev[s][0].record(stream)
            ctx.evaluate(R, out=out)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        ctx.close()
        return ms

    # distinct determinants of every |c|-ordered prefix: count first occurrences along the order
    order = np.argsort(-np.abs(wl.ci_coef), kind="stable")
    prefix = []
    for D in (wl.det_up, wl.det_dn):
        _, ids = np.unique(D, axis=0, return_inverse=True)
        ids = ids.ravel()[order]
        first = np.zeros(len(ids), bool)
        _, pos = np.unique(ids, return_index=True)
        first[pos] = True
        prefix.append(np.cumsum(first))
    rows = []
    with ClockSampler(_gpu_index(0)) as clk:
        full_ms = timed(np.ones(len(wl.ci_coef), bool))
        for eps in (1e-7, 1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13):
            keep, _, _, cnt = pkg.truncate_norm(wl.det_up, wl.det_dn, wl.ci_coef, eps, eps)
            # the longest |c| prefix whose distinct determinants do not exceed the norm truncation's
            n_c = int(np.searchsorted(prefix[0] + prefix[1], cnt["up"] + cnt["dn"], side="right"))
            cmask = np.zeros(len(order), bool)
            cmask[order[:n_c]] = True
            rows.append({"eps": eps,
                         "norm": {"products": cnt["products"], "up": cnt["up"], "dn": cnt["dn"],
                                  "norm_lost": 1.0 - float(np.sum(wl.ci_coef[keep] ** 2)) / total,
                                  "walker_steps_per_s": wl.n_walk / (timed(keep) / 1e3)},
                         "coef": {"products": n_c, "up": int(prefix[0][n_c - 1]), "dn": int(prefix[1][n_c - 1]),
                                  "c_min": float(abs(wl.ci_coef[order[n_c - 1]])),
                                  "norm_lost": 1.0 - float(np.sum(wl.ci_coef[cmask] ** 2)) / total,
                                  "walker_steps_per_s": wl.n_walk / (timed(cmask) / 1e3)}})
    line = {"metric": "walker-steps/s vs truncation threshold, norm-based vs |c| truncation (Table 5 analogue)",
            "value": wl.n_walk / (full_ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": full_ms, "higher_is_better": True,
            "dtype": "f64+f32x2" if prec == pkg.PRECISION_MIXED else "f64", "data": "synthetic",
            "config": {"workload": "truncation_750k", "precision": args.precision, "walkers": wl.n_walk,
                       "n_det": int(len(wl.ci_coef)), "l2": "flushed between timed steps"},
            "rows": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_sm_chain(args):
    """The paper's sequential Sherman-Morrison chain (Sec. 2.2) against the
    table method on the 750k expansion (8,192 walkers, FP64 orbitals of one
    evaluation): ms per step for the chain (both spins) and for the table
    method's reference + ratio stages, the chain's N_inv and N_subst per
    walker-step (Table 3), and the relative difference of the two sets of ratios
    on 64 sampled walkers."""
    import numpy as np
    import torch

    import paper_1510_00730_gb300 as pkg
    from paper_1510_00730_gb300 import costs, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    wl = synth.chlorine_like_750k()
    ctx = pkg.Context.from_workload(wl, device=0, precision=pkg.PRECISION_FP64)
    R = torch.from_numpy(wl.R).to(dev)
    out = ctx.alloc_outputs(wl.n_walk)
    ctx.set_profiling(True)
    stream = torch.cuda.current_stream(dev)
    stages = []
    for s in range(args.warmup + args.steps):
        ctx.evaluate(R, out=out)
        torch.cuda.synchronize()
        if s >= args.warmup:
            stages.append(ctx.profile())
    table_ms = statistics.mean(p["reference"] + p["ratios"] for p in stages)
    ev = []
    with ClockSampler(_gpu_index(0)) as clk:
        for s in range(args.warmup + args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r, n_inv, n_subst = ctx.sm_chain(wl.n_walk)
            b.record(stream)
            if s >= args.warmup:
                ev.append((a, b))
        torch.cuda.synchronize()
    chain_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    st = ctx.stats()
    r_up, r_dn, _, _ = ctx.ratios(wl.n_walk)
    table = np.concatenate([r_up, r_dn], axis=1)
    chain = r.cpu().numpy()[:, :wl.n_walk].T
    idx = np.arange(0, wl.n_walk, wl.n_walk // 64)
    diff = np.abs(chain[idx] - table[idx]) / np.maximum(np.abs(table[idx]), 1.0)
    line = {"metric": "ms per step of the determinant ratios: sequential Sherman-Morrison chain vs table method",
            "value": chain_ms, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": chain_ms, "higher_is_better": False, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "sm_chain_750k", "walkers": wl.n_walk, "n_det_up": st["n_det_up"],
                       "n_det_dn": st["n_det_dn"], "threshold": 1e-3},
            "table_ms": table_ms, "chain_over_table": chain_ms / table_ms,
            "n_inv": float(n_inv.double().mean()), "n_subst": float(n_subst.double().mean()),
            # per distinct determinant, and what a fixed reference would need (Sec. 5's 1.78 against 3.46)
            "n_subst_per_det": float(n_subst.double().mean()) / (st["n_det_up"] + st["n_det_dn"]),
            "n_subst_per_det_fixed_reference": costs.fixed_reference_substitutions(
                *[np.bincount(ctx.spin_dets(sp)[1]) for sp in (0, 1)]),
            "ratio_difference": {"p50": float(np.median(diff)), "p99": float(np.percentile(diff, 99)),
                                 "max": float(diff.max())},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_learned(args):
    """The learned Metropolis proposal on the chlorine-like 10^5-determinant
    expansion with 8,192 walkers: a chain of drift-diffusion moves (limited
    drift) generates 2^20 configurations, the perceptron is trained on them
    on the GPU (generalised speed measure), and both movers then run the same
    number of steps from the same walkers. value = autocorrelation-corrected
    samples/s of <E_L> with the learned move (walker-steps/s / tau_int(E_L),
    Sokal window c = 5); the drift-diffusion chain is reported beside it."""
    import torch

    import paper_1510_00730_gb300 as pkg
    from paper_1510_00730_gb300 import synth
    from paper_1510_00730_gb300.vmc import learned_vs_drift_diffusion
    torch.cuda.set_device(0)
    wl = synth.chlorine_like_100k(n_walk=8192)
    prec = {"mixed": pkg.PRECISION_MIXED, "fp64": pkg.PRECISION_FP64}[args.precision]
    ctx = pkg.Context.from_workload(wl, device=0, precision=prec)
    tau = 3e-5
    n_chain = max(args.steps, 100)
    with ClockSampler(_gpu_index(0)) as clk:
        r = learned_vs_drift_diffusion(ctx, wl.R, tau, n_chain, warmup=args.warmup)
    learned = r["learned"]
    line = {"metric": "autocorrelation-corrected samples/s of <E_L>, learned proposal vs drift-diffusion",
            "value": learned["samples_per_s"], "unit": "samples/s", "n_gpus": 1, "steps": n_chain,
            "warmup": args.warmup, "ms_per_step": learned["ms_per_step"], "higher_is_better": True,
            "dtype": "f64+f32x2" if prec == pkg.PRECISION_MIXED else "f64", "data": "synthetic",
            "config": {"workload": "learned_proposal_100k", "walkers": wl.n_walk, "n_det": int(wl.n_det),
                       "tau": tau, "drift_limit_a": 1.0, "training_configs": r["training_configs"],
                       "mlp": "51-256-256-68 tanh on tcgen05 tensor cores: BF16 weights and activations, "
                              "FP32 accumulation",
                       "objective": "generalised speed measure, target acceptance 0.5"},
            "learned": learned, "drift_diffusion": r["drift_diffusion"],
            "drift_diffusion_limited": r["drift_diffusion_limited"],
            "gain": r["gain"], "gain_err": r["gain_err"], "gain_vs_limited": r["gain_vs_limited"],
            "gain_vs_limited_err": r["gain_vs_limited_err"],
            "training": {"collect_s": r["collect_s"], "train_s": r["train_s"],
                         "objective_acceptance_per_epoch": r["objective_acceptance_per_epoch"]},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="chlorine_like_750k")
    p.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--no-compare", dest="compare", action="store_false",
                   help="skip timing the other precision in the same run")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batch", dest="batch", action="store_false",
                   help="skip the 64-expansion graph batch that the default line reports beside the headline")
    p.add_argument("--chunks", type=int, default=None, help="walker chunks of the mixed path (default: library's)")
    p.add_argument("--fallback-tol", type=float, default=None,
                   help="fallback tolerance of the timed contexts (default: the library's, 1e-5 mixed, 1e-8 FP64)")
    p.add_argument("--streams", type=int, default=8, help="streams of the batched workload")
    p.add_argument("--tune-ms", type=float, default=60.0, help="autotuner budget per expansion (batched workload)")
    p.add_argument("--ref-sample", type=int, default=32)
    p.add_argument("--traffic", type=float, default=None, help="DRAM bytes per launch of the dominant kernel (ncu)")
    args = p.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched_uneven_64":
        run_batched(args)
    elif args.workload == "learned_proposal_100k":
        run_learned(args)
    elif args.workload == "truncation_750k":
        run_truncation(args)
    elif args.workload == "sm_chain_750k":
        run_sm_chain(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
