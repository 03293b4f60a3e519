"""Benchmark of the fused propagate + Kalman-update kernels on GB300.

One step = the whole hot path over one batch: p2r on 100 events x 9600 tracks
x 20 cylinders (one launch) and p2z on 100 x 9600 x 20 planes (one launch).
Metric: track-layer propagate+update per second (kernel time, inputs resident
in HBM).  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs under torchrun, one rank per GPU; every rank fits its own batch of
the same size (weak scaling, no data exchange) and rank 0 reports the
whole-job throughput over the slowest rank's time.  --impl reference times the
FP64 CPU oracle on the host cores over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NEVT, NTRK, NLAYER, SEED = 100, 9600, 20, 2
# The headline metric: track-layers per second (the value), reported with the
# roofline fraction and the CPU oracle beside it.
METRIC = "track-layer propagate+update/s on 1 GB300; % of FP32/HBM roofline vs oracle"
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0
MUFU_LANES_PER_SM = 16

# Algorithmic work per track-layer: a fixed count of the FP32 operations of
# the method's formulas (FMA = 2), the same for every build of the kernel, so
# that a leaner kernel raises the roofline fraction instead of lowering it.
#   p2z: helix to the plane ~30, Jacobian and J C J^T (sparse) ~330, 2-D
#        Kalman update (gain, state, covariance, chi2) ~220: 580.
#   p2r: ~600 outside the path-length iteration, ~50 per iteration (helix at
#        h and the straight-line step to the cylinder); the iterations per
#        track-layer are counted by the kernel on every run.
# MUFU (sin/cos, square root, reciprocal) operations per track-layer: p2z 3
# sin/cos + 1 reciprocal; p2r 1 sin/cos + 1 atan2 or rsqrt + per iteration 1
# sin/cos + 1 square root.
FLOPS_P2Z = 580.0
FLOPS_P2R_FIXED = 600.0
FLOPS_P2R_PER_ITERATION = 50.0
MUFU_P2Z = 4.0


def flops_p2r(iterations: float) -> float:
    return FLOPS_P2R_FIXED + FLOPS_P2R_PER_ITERATION * iterations


def mufu_p2r(iterations: float) -> float:
    return 2.0 + 2.0 * iterations


BYTES_TRACK_IN = (6 + 21 + 1) * 4
BYTES_TRACK_OUT = (6 + 21 + 1 + 1) * 4 + 1


def set_nevt(n: int) -> None:
    global NEVT
    NEVT = n


# Hit bytes a track-layer needs: p2r measures the azimuthal coordinate and z
# (all 3 positions and 6 covariance entries); p2z measures (x, y) on the
# plane (2 positions, the 3 (x, y) covariance entries).
HIT_BYTES = (36.0, 20.0)


def bytes_per_track_layer(nlayer: int, mode: int = 0) -> float:
    return HIT_BYTES[mode] + (BYTES_TRACK_IN + BYTES_TRACK_OUT) / nlayer


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured",
                "sm_max_mhz": float(d.get("sm_max_mhz", SM_MAX_MHZ_NOMINAL))}
    return {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": SM_MAX_MHZ_NOMINAL}


def fp32_peak_tflops(mhz: float, sms: int) -> float:
    """FP32 ceiling from unit counts: SMs x 128 FP32 lanes x 2 flops x clock."""
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def mufu_peak_tops(mhz: float, sms: int) -> float:
    return sms * MUFU_LANES_PER_SM * mhz * 1e6 / 1e12


def sm_count(local: int) -> int:
    import torch
    return int(torch.cuda.get_device_properties(local).multi_processor_count)


def measure_fp32(local: int) -> dict:
    """The FP32 throughput probe (fit_probe_fp32) on this device, scalar and
    packed FMAs, with the SM clock sampled while it runs: checks the derived
    FP32 ceiling against the hardware."""
    import torch
    from paper_2409_09228_gb300 import fit
    dev = torch.device("cuda", local)
    sms = sm_count(local)
    blocks = sms * 8 * 4  # 8 resident blocks of 256 per SM, 4 waves
    out = torch.empty(blocks * fit.FIT_PROBE_THREADS, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.2)
    for packed, name in ((0, "ffma"), (1, "ffma2")):
        iters = 2048 if packed else 4096
        for _ in range(2):
            fit.fit_probe_fp32(packed, blocks, iters, out, stream)
        best = float("inf")
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            flops = fit.fit_probe_fp32(packed, blocks, iters, out, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            best = min(best, e0.elapsed_time(e1))
        res[f"{name}_tflops"] = flops / (best / 1e3) / 1e12
    clk = clocks.stop()
    res["sm_mhz"] = clk["sm_mhz"]
    res["sms"] = sms
    if clk["sm_mhz"]:
        res["derived_at_this_clock_tflops"] = fp32_peak_tflops(clk["sm_mhz"], sms)
    return res


# The sources fit_fused_kernel is compiled from (and the constants it takes
# from include/fit.h): a DRAM traffic figure measured by ncu holds only while
# their code (comments and layout aside) hashes to the value stored with it.
FUSED_SOURCES = ("paper_2409_09228_gb300/csrc/fit.cu",
                 "paper_2409_09228_gb300/csrc/fused.cuh",
                 "paper_2409_09228_gb300/csrc/track_math.cuh",
                 "paper_2409_09228_gb300/csrc/lanes.cuh",
                 "paper_2409_09228_gb300/csrc/internal.h")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")


def code_only(text: str) -> str:
    """C++ source without its comments and with whitespace runs collapsed, so
    that editing a comment or re-wrapping a line keeps the hash."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":  # a literal: copied up to its closing quote
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in FUSED_SOURCES:
        with open(os.path.join(ROOT, name)) as f:
            h.update(name.encode() + code_only(f.read()).encode())
    with open(os.path.join(ROOT, "include", "fit.h")) as f:
        h.update("".join(l for l in f if l.startswith("#define FIT_")).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str) -> float | None:
    """DRAM bytes (read + write) per launch of `kernel` on this workload, as
    ncu measured them, if they were measured on the current source."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        entries = json.load(f)
    e = entries.get(f"{kernel}_{NEVT}x{NTRK}x{NLAYER}")
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_launch"])


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                mhz.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def dist_setup(gpus: int, backend: str | None = None):
    """Rank, world size and local rank from the torchrun environment; for
    N > 1 one process group (NCCL on GPUs, gloo without).  Every rank fits its
    own batch: there is no data exchange, only the barrier around the timed
    region and the maximum of the ranks' times."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


_WORKLOAD = {}


def workload(rank: int):
    """The rank's own batch (weak scaling): both modes, NEVT x NTRK tracks,
    drawn from seed SEED + 1000 rank (generated once per process)."""
    from paper_2409_09228_gb300 import inputs
    key = (rank, NEVT, NTRK, NLAYER)
    if key not in _WORKLOAD:
        n = NEVT * NTRK
        _WORKLOAD[key] = [inputs.generate(m, n, seed=SEED + 1000 * rank, nlayer=NLAYER)
                          for m in (0, 1)]
    return _WORKLOAD[key]


def cpu_baseline(sets, budget_s: float = 12.0) -> dict:
    """The FP64 oracle on the host cores over whole events, until budget_s elapses."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    done, t0 = 0, time.perf_counter()
    evts = 0
    while evts < NEVT and time.perf_counter() - t0 < budget_s:
        for ts in sets:
            sub = ts.subset(np.arange(evts * NTRK, (evts + 1) * NTRK))
            oracle.fit_set(sub, nthreads=cores)
            done += NTRK * NLAYER
        evts += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "track-layer/s", "cores": cores, "kind": "oracle",
            "sample": f"{evts} of {NEVT} events of each mode (p2r + p2z, {NTRK} tracks x "
                      f"{NLAYER} layers each), FP64, {dt:.1f} s"}


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    from paper_2409_09228_gb300 import inputs
    cores = len(os.sched_getaffinity(0))
    ev_per_step = 1
    sets = [inputs.generate(m, ev_per_step * NTRK, seed=SEED, nlayer=NLAYER) for m in (0, 1)]
    for _ in range(args.warmup):
        for ts in sets:
            oracle.fit_set(ts, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for ts in sets:
            oracle.fit_set(ts, nthreads=cores)
    dt = (time.perf_counter() - t0) / args.steps
    units = 2 * ev_per_step * NTRK * NLAYER
    v = units / dt
    line = {"impl": "reference", "metric": METRIC,
            "value": v, "unit": "track-layer/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": "track-layer/s",
                             "sample": f"{ev_per_step} event of each mode per step "
                                       f"({units} track-layers)"},
            "e2e": {"value": v, "unit": "track-layer/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def config_dict(args):
    return {"workload": f"p2r + p2z fused fit, {NEVT} events x {NTRK} tracks x {NLAYER} layers "
                        f"per mode, one launch per mode",
            "nevt": NEVT, "ntrk": NTRK, "nlayer": NLAYER, "modes": ["p2r", "p2z"],
            "global_batch": args.gpus * 2 * NEVT * NTRK, "parallelism": f"dp{args.gpus}",
            "l2": "inputs larger than L2 (691 MB of hits per mode per step); no flush"}


def bench_uneven(args, world, rank, local):
    """2000 events, log-normal track counts (median 2000, sigma 1, clipped
    50..20000), p2r or p2z at random per event, 20 layers: the per-segment
    path (one launch per run of same-mode events) against the batched
    persistent plan (one launch under a CUDA graph), default and autotuned."""
    import torch
    from paper_2409_09228_gb300 import fit, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nevt = args.uneven_events
    nt = inputs.uneven_event_sizes(nevt, 3)
    md = inputs.uneven_event_modes(nevt, 3)
    ev = inputs.generate_events(nt, md, seed=3 + 1000 * rank)
    n = ev.n
    ld = (n + 31) // 32 * 32  # AoSoA-ready: the tuner may choose either layout
    up = lambda a: torch.from_numpy(np.ascontiguousarray(np.pad(a, [(0, 0)] * (a.ndim - 1) + [(0, ld - n)]))).to(dev)  # noqa: E731
    dev_in = [up(a) for a in (ev.par0, ev.cov0, ev.q, ev.hpos, ev.hcov)]
    del ev.hpos, ev.hcov
    f = fit.Fitter(fit.Geometry(ev.B, ev.surf[0]), fit.Geometry(ev.B, ev.surf[1]), device=local)
    out = f.outputs(n, ld=ld)
    stream = torch.cuda.current_stream(dev)
    bufs = dict(par_out=out["par"], cov_out=out["cov"], q_out=out["q"], chi2=out["chi2"],
                status=out["status"])

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(world, e0.elapsed_time(e1) / args.steps)

    seg_ms = timed(lambda: f.run(*dev_in, nt, md, out=out, stream=stream))
    plan = fit.fit_plan_create(f.h, nt, md, NLAYER, layout=fit.FIT_LAYOUT_TUNE)
    plan_ms = timed(lambda: fit.fit_plan_run(plan, *dev_in, stream=stream, **bufs))
    info_default = fit.fit_plan_get_info(plan)
    t0 = time.perf_counter()
    info = fit.fit_plan_tune(plan, *dev_in, stream=stream, **bufs)
    tune_s = time.perf_counter() - t0
    if info["layout"] == fit.FIT_LAYOUT_AOSOA32:  # the caller's arrays, converted once
        conv = []
        for k, a in enumerate(dev_in):
            if k == 2:
                conv.append(a)
                continue
            b = torch.empty_like(a)
            fit.fit_relayout(a, fit.FIT_LAYOUT_SOA, b, fit.FIT_LAYOUT_AOSOA32, stream=stream)
            conv.append(b)
        dev_in = conv
    tuned_ms = timed(lambda: fit.fit_plan_run(plan, *dev_in, stream=stream, **bufs))
    st = f.sync(stream)
    assert st["nonfinite"] == 0 and st["no_intersection"] == 0, st
    fit.fit_plan_destroy(plan)
    f.close()
    if rank != 0:
        return
    units = world * n * NLAYER
    segments = int(1 + np.count_nonzero(np.diff(md)))
    line = {"metric": "track-layer propagate+update/s", "value": units / (tuned_ms / 1e3),
            "unit": "track-layer/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tuned_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"uneven batch: {nevt} events, log-normal track counts "
                                   f"(median 2000, sigma 1, 50..20000), p2r/p2z per event, "
                                   f"{NLAYER} layers", "tracks": n, "events": nevt,
                       "same_mode_runs": segments},
            "per_segment_launches": {"ms": seg_ms, "launches": segments,
                                     "value": units / (seg_ms / 1e3)},
            "plan_default": {"ms": plan_ms, "value": units / (plan_ms / 1e3), **info_default},
            "plan_tuned": {"ms": tuned_ms, "tuning_s": tune_s, **info}}
    return line


def bench_adjoint(args, world, rank, local):
    """Gradient of the summed chi2 w.r.t. hit positions and initial parameters
    for 100k p2r tracks x 20 layers (forward with per-layer checkpoints, then
    the reverse sweep), against the FP64 oracle's dual-number gradient timed on
    the host cores over a sample."""
    import torch
    from paper_2409_09228_gb300 import fit, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n = args.adjoint_tracks
    ts = inputs.generate(inputs.MODE_R, n, seed=5 + 1000 * rank)
    ld = (n + 3) // 4 * 4
    up = lambda a: torch.from_numpy(np.ascontiguousarray(np.pad(a, [(0, 0)] * (a.ndim - 1) + [(0, ld - n)]))).to(dev)  # noqa: E731
    d = [up(a) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    f = fit.Fitter(fit.Geometry(ts.B, ts.surf), None, device=local)
    tape = torch.empty(fit.fit_tape_bytes(NLAYER, ld) // 4, device=dev)
    out = f.outputs(n, ld=ld)
    w = torch.ones(ld, device=dev)
    gh = torch.empty_like(d[3])
    gp = torch.empty((6, ld), device=dev)
    gc = torch.empty((21, ld), device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        fit.fit_adjoint_forward(f.h, *d, [n], [0], tape, out["par"], out["cov"], out["q"],
                                out["chi2"], stream=stream)
        fit.fit_adjoint_backward(f.h, d[3], d[4], [n], [0], tape, w, gh, gp, gc, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps)
    f.sync(stream)
    f.close()
    if rank != 0:
        return
    line = {"metric": "track-layer chi2-gradient/s", "value": world * n * NLAYER / (ms / 1e3),
            "unit": "track-layer/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"adjoint: d(sum chi2)/d(hit positions, initial parameters), "
                                   f"{n} p2r tracks x {NLAYER} layers, per-layer checkpoints",
                       "tape_bytes": fit.fit_tape_bytes(NLAYER, ld)}}
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = len(os.sched_getaffinity(0))
        m = 2000
        sub = ts.subset(np.arange(m))
        t0 = time.perf_counter()
        oracle.chi2_grad(sub.mode, sub.B, sub.surf, sub.par0, sub.cov0, sub.q, sub.hpos, sub.hcov,
                         nthreads=cores)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": m * NLAYER / dt, "unit": "track-layer/s", "cores": cores,
                                "kind": "oracle", "sample": f"{m} of {n} tracks, FP64 dual numbers, {dt:.1f} s"}
    return line


FP64_PEAK_TFLOPS_NOMINAL = 1.25  # GB300 FP64 (non-tensor), nominal; no measured figure


def bench_f64(args, world, rank, local):
    """The FP64 variant on the bench workload (100 events x 9600 tracks x 20
    layers per mode, double buffers, one launch per mode): what double costs
    on GB300, whose FP64 rate is a small fraction of its FP32 rate."""
    import torch
    from paper_2409_09228_gb300 import fit

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sets = workload(rank)
    # a double fit: the p2r iteration to 1e-12 R
    f = fit.Fitter(fit.Geometry(sets[0].B, sets[0].surf, tol=1e-12),
                   fit.Geometry(sets[1].B, sets[1].surf, tol=1e-12), device=local)
    n = NEVT * NTRK
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a.astype(np.float64) if a.dtype.kind == "f" else a)).to(dev)  # noqa: E731
    d_in = [[up(a) for a in (s.par0, s.cov0, s.q, s.hpos, s.hcov)] for s in sets]
    outs = [{"par": torch.empty((6, n), dtype=torch.float64, device=dev),
             "cov": torch.empty((21, n), dtype=torch.float64, device=dev),
             "q": torch.empty(n, dtype=torch.int32, device=dev),
             "chi2": torch.empty(n, dtype=torch.float64, device=dev)} for _ in sets]
    stream = torch.cuda.current_stream(dev)
    ntrk = [NTRK] * NEVT
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(2)]
    kern = [[], []]

    def step(record=False):
        for m in (0, 1):
            if record:
                ev[m][0].record(stream)
            o = outs[m]
            fit.fit_propagate_update_f64(f.h, *d_in[m], ntrk, [m] * NEVT, o["par"], o["cov"],
                                         o["q"], o["chi2"], stream=stream)
            if record:
                ev[m][1].record(stream)

    clocks = ClockSampler(local)  # started before the warm-up, as in the headline
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step()
    st = f.sync(stream)
    assert st["nonfinite"] == 0 and st["no_intersection"] == 0, st
    torch.cuda.synchronize(dev)
    barrier(world)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
        torch.cuda.synchronize(dev)
        for m in (0, 1):
            kern[m].append(ev[m][0].elapsed_time(ev[m][1]))
    t1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = max_over_ranks(world, sum(statistics.mean(k) for k in kern))
    st = f.sync(stream)
    f.close()
    if rank != 0:
        return
    tl = n * NLAYER
    kms = [statistics.mean(k) for k in kern]
    it_f64 = st["iterations"] / (args.steps * tl)
    ach = flops_p2r(it_f64) * tl / (kms[0] / 1e3) / 1e12
    line = {"metric": "track-layer propagate+update/s", "value": world * 2 * tl / (ms / 1e3),
            "unit": "track-layer/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"FP64 variant: p2r + p2z, {NEVT} events x {NTRK} tracks x "
                                   f"{NLAYER} layers per mode, double buffers, one launch per mode, "
                                   f"p2r iteration to 1e-12 R",
                       "inputs_exceed_l2": True},
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS_NOMINAL,
                         "unit": "TFLOP/s (FP64)", "frac": ach / FP64_PEAK_TFLOPS_NOMINAL,
                         "peak_source": "nominal GB300 FP64 rate", "traffic": None,
                         "kernel": "fit_f64_kernel<p2r>", "kernel_ms_p2r_p2z": kms,
                         "flops_per_track_layer": flops_p2r(it_f64)},
            "clocks": clk, "gpu_launches": 2 * args.steps,
            "p2r_iterations_per_track_layer": st["iterations"] / (args.steps * tl)}
    return line


def bench_layout(args, world, rank, local):
    """Ablation of the track and hit layout on the bench workload: structure
    of arrays (the default path) against the paper's AoSoA with tiles of 32
    tracks (fit_propagate_update_layout), same kernels otherwise."""
    import torch
    from paper_2409_09228_gb300 import fit, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sets = workload(rank)
    f = fit.Fitter(fit.Geometry(sets[0].B, sets[0].surf), fit.Geometry(sets[1].B, sets[1].surf),
                   device=local)
    n = NEVT * NTRK
    ld = (n + 31) // 32 * 32
    stream = torch.cuda.current_stream(dev)
    ntrk = [NTRK] * NEVT
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    res = {}
    for name, layout in (("soa", fit.FIT_LAYOUT_SOA), ("aosoa32", fit.FIT_LAYOUT_AOSOA32)):
        conv = (lambda a: up(a)) if layout == fit.FIT_LAYOUT_SOA else \
            (lambda a: up(inputs.to_aosoa32(a, ld)))
        d = [[conv(a) for a in (s.par0, s.cov0)] + [up(np.pad(s.q, (0, ld - n)))] +
             [conv(a) for a in (s.hpos, s.hcov)] for s in sets]
        o = [{"par": torch.empty(6 * ld, device=dev), "cov": torch.empty(21 * ld, device=dev),
              "q": torch.empty(ld, dtype=torch.int32, device=dev),
              "chi2": torch.empty(ld, device=dev)} for _ in sets]
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(2)]
        kern = [[], []]
        for k in range(args.warmup + args.steps):
            for m in (0, 1):
                ev[m][0].record(stream)
                fit.fit_propagate_update_layout(f.h, *d[m], ntrk, [m] * NEVT, layout, ld,
                                                o[m]["par"], o[m]["cov"], o[m]["q"], o[m]["chi2"],
                                                stream=stream)
                ev[m][1].record(stream)
            torch.cuda.synchronize(dev)
            if k >= args.warmup:
                for m in (0, 1):
                    kern[m].append(ev[m][0].elapsed_time(ev[m][1]))
        st = f.sync(stream)
        assert st["nonfinite"] == 0 and st["no_intersection"] == 0, st
        kms = [statistics.median(x) for x in kern]
        res[name] = {"p2r_ms": kms[0], "p2z_ms": kms[1],
                     "value": world * 2 * n * NLAYER / (sum(kms) / 1e3)}
        del d, o
    f.close()
    if rank != 0:
        return
    ms = res["aosoa32"]["p2r_ms"] + res["aosoa32"]["p2z_ms"]
    line = {"metric": "track-layer propagate+update/s", "value": res["aosoa32"]["value"],
            "unit": "track-layer/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"layout ablation: p2r + p2z, {NEVT} events x {NTRK} tracks x "
                                   f"{NLAYER} layers per mode, AoSoA tiles of 32 tracks against "
                                   f"structure of arrays", "inputs_exceed_l2": True},
            "layouts": res, "gpu_launches": 2 * (args.warmup + args.steps) * 2}
    return line


def bench_find(args, world, rank, local):
    """Track finding: NEVT/4 events x 9600 tracks x 20 layers per mode, 4
    candidate hits per layer (the track's own with probability 0.95, noise
    displaced by 20 hit errors), chi2 gate 30, FP32, one launch per mode."""
    import torch
    from paper_2409_09228_gb300 import fit, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    nevt, ncand = max(1, NEVT // 4), 4
    n = nevt * NTRK
    sets = [inputs.generate(m, n, seed=SEED + 1000 * rank, nlayer=NLAYER) for m in (0, 1)]
    cands = [inputs.generate_candidates(s, ncand, seed=SEED + 1000 * rank, spread=20.0) for s in sets]
    f = fit.Fitter(fit.Geometry(sets[0].B, sets[0].surf), fit.Geometry(sets[1].B, sets[1].surf),
                   device=local)
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    d = [[up(a) for a in (s.par0, s.cov0, s.q, c.cpos, c.ccov)] for s, c in zip(sets, cands)]
    for s, c in zip(sets, cands):
        del s.hpos, s.hcov, c.cpos, c.ccov
    o = [[torch.empty((6, n), device=dev), torch.empty((21, n), device=dev),
          torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, device=dev)] for _ in sets]
    chosen = [torch.empty((NLAYER, n), dtype=torch.int8, device=dev) for _ in sets]
    stream = torch.cuda.current_stream(dev)
    ntrk = [NTRK] * nevt
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(2)]
    kern = [[], []]
    for k in range(args.warmup + args.steps):
        for m in (0, 1):
            ev[m][0].record(stream)
            fit.fit_find_tracks(f.h, *d[m], ntrk, [m] * nevt, 30.0, chosen[m], *o[m],
                                stream=stream)
            ev[m][1].record(stream)
        torch.cuda.synchronize(dev)
        if k >= args.warmup:
            for m in (0, 1):
                kern[m].append(ev[m][0].elapsed_time(ev[m][1]))
    st = f.sync(stream)
    taken = float((chosen[0] >= 0).float().mean().item())
    f.close()
    kms = [statistics.median(x) for x in kern]
    ms = max_over_ranks(world, sum(kms))
    if rank != 0:
        return
    tl = n * NLAYER
    peaks = load_peaks()
    bpl = 36.0 * ncand + 1.0 + (BYTES_TRACK_IN + BYTES_TRACK_OUT - 1) / NLAYER
    ach = bpl * tl / (kms[0] / 1e3) / 1e9
    line = {"metric": "track-layer propagate+find+update/s", "value": world * 2 * tl / (ms / 1e3),
            "unit": "track-layer/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"track finding: p2r + p2z, {nevt} events x {NTRK} tracks x "
                                   f"{NLAYER} layers per mode, {ncand} candidate hits per layer, "
                                   f"chi2 gate 30", "inputs_exceed_l2": True},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / peaks["hbm_gbs"], "traffic": None,
                         "kernel": "fit_find_kernel<p2r, float>", "bytes_per_track_layer": bpl,
                         "kernel_ms_p2r_p2z": kms},
            "gpu_launches": 2 * (args.warmup + args.steps), "p2r_layers_with_a_hit": taken,
            "status": st}
    return line


def bench_seed(args, world, rank, local):
    """The learned p2r path-length seed.  Trains the network on 4M single p2r
    propagations labelled by the library's own exact iteration (run to
    1e-7 R), then fits 1M p2r tracks x 20 layers with the straight-line start
    (the packed two-tracks-per-thread kernel), with the network (one track
    per thread, the network before every layer) and with the closed-form
    crossing start (packed kernel), and times the path-length step alone on
    4M states with each start.  The value is the seeded fit's throughput; the
    line carries the other two beside it."""
    import torch
    from paper_2409_09228_gb300 import fit, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    surf = inputs.surfaces(inputs.MODE_R)

    # training data: exact path lengths from the iteration itself, tight tolerance
    lab = fit.Fitter(fit.Geometry(inputs.B_FIELD, surf, max_iter=30, tol=1e-7), None, device=local)

    def labelled(nsamp, seed):
        ss = inputs.seed_samples(nsamp, seed=seed)
        par, q, R = up(ss.par), up(ss.q), up(ss.R)
        h = torch.empty(nsamp, device=dev)
        fit.fit_path_lengths(lab.h, par, q, R, h, stream=stream)
        x = torch.empty((nsamp, 8), device=dev)
        t = torch.empty(nsamp, device=dev)
        fit.fit_mlp_prepare(ss.B, par, q, R, x, h_exact=h, target=t, stream=stream)
        return ss, par, q, R, h, x, t

    _, _, _, _, _, x, t = labelled(args.seed_train_samples, 4)
    m = fit.fit_mlp_create(local, seed=4)
    t0 = time.perf_counter()
    curve = fit.fit_mlp_train(m, x, t, epochs=args.seed_epochs, batch=4096, lr=2e-3,
                              lr_final=1e-6, seed=4, stream=stream)
    train_s = time.perf_counter() - t0
    del x, t
    # the network replaces the straight-line start; fc starts at the closed-form crossing
    f = fit.Fitter(fit.Geometry(inputs.B_FIELD, surf, start=fit.FIT_START_LINE), None,
                   device=local)
    fc = fit.Fitter(fit.Geometry(inputs.B_FIELD, surf, start=fit.FIT_START_CROSSING), None,
                    device=local)
    fit.fit_mlp_attach(f.h, m, stream=stream)
    # the path-length step alone, held-out states
    ss, par, q, R, h_ex, xe, _ = labelled(4_000_000, 400 + 1000 * rank)
    ye = torch.empty(ss.n, device=dev)
    fit.fit_mlp_forward(m, xe, ye, stream=stream)
    hl = torch.empty(ss.n, device=dev)
    its = torch.empty(ss.n, dtype=torch.int32, device=dev)

    def step_alone(fitter, seeded):
        fit.fit_path_lengths(fitter.h, par, q, R, hl, its, seeded=seeded, stream=stream)

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    alone = {}
    for label, fitter, seeded in (("straight_line", f, False), ("network", f, True),
                                  ("crossing", fc, False)):
        ms = timed(lambda: step_alone(fitter, seeded), args.steps)
        alone[label] = {
            "ms": ms, "iterations_per_state": float(its.double().mean().item()),
            "one_iteration": float((its == 1).double().mean().item()),
            "max_abs_dh_vs_1e-7_iteration_cm": float((hl - h_ex).abs().max().item())}
    seed_err = None
    # seed error of the held-out states in units of the tolerance 1e-6 R
    with torch.no_grad():
        kB = inputs.KA * float(np.float32(inputs.B_FIELD))
        x0, y0, ph = par[0].double(), par[1].double(), par[4].double()
        b = x0 * torch.cos(ph) + y0 * torch.sin(ph)
        c = x0 * x0 + y0 * y0 - R.double() ** 2
        hline = -b + torch.sqrt(b * b - c)
        kap = -q.double() * kB * par[3].double()
        hs = hline + ye.double() * 0.5 * kap * hline * hline
        e = ((hs - h_ex.double()).abs() / (1e-6 * R.double())).cpu().numpy()
        seed_err = {"median_over_tol": float(np.median(e)), "within_tol": float(np.mean(e <= 1)),
                    "p99_over_tol": float(np.quantile(e, 0.99))}
    del xe, ye, hl, its, par, q, R, h_ex
    lab.close()

    # the fit: 1M tracks x 20 layers, plain and seeded
    n = args.seed_tracks
    ts = inputs.generate(inputs.MODE_R, n, seed=4 + 1000 * rank)
    ld = (n + 3) // 4 * 4
    pad = lambda a: up(np.pad(a, [(0, 0)] * (a.ndim - 1) + [(0, ld - n)]))  # noqa: E731
    d = [pad(a) for a in (ts.par0, ts.cov0, ts.q, ts.hpos, ts.hcov)]
    out = f.outputs(n, ld=ld)
    res = {}
    clk = None
    for label, fitter, net in (("straight_line", f, None), ("network", f, m),
                               ("crossing", fc, None)):
        fit.fit_mlp_attach(fitter.h, net, stream=stream)
        if net is not None:  # started before the warm-up, as in the headline
            clocks = ClockSampler(local)
            clocks.start()
            time.sleep(0.3)
        for _ in range(args.warmup):
            fitter.run(*d, [n], [0], out=out, stream=stream)
        fitter.sync(stream)
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fitter.run(*d, [n], [0], out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if net is not None:
            clk = clocks.stop()
        st = fitter.sync(stream)
        assert st["nonfinite"] == 0 and st["no_intersection"] == 0 and st["not_converged"] == 0, st
        ms = max_over_ranks(world, e0.elapsed_time(e1) / args.steps)
        res[label] = {"ms": ms, "value": world * n * NLAYER / (ms / 1e3),
                      "iterations_per_track_layer": st["iterations"] / (args.steps * n * NLAYER)}
    f.close()
    fc.close()
    fit.fit_mlp_destroy(m)
    if rank != 0:
        return
    ms = res["network"]["ms"]
    tl = n * NLAYER
    peaks = load_peaks()
    alu_peak = fp32_peak_tflops(peaks["sm_max_mhz"], sm_count(local))
    seeded_flops = flops_p2r(res["network"]["iterations_per_track_layer"])
    alu_ach = seeded_flops * tl / (ms / 1e3) / 1e12
    mlp_flops = 2.0 * 4801  # multiply-adds of the network per track-layer, x 2
    line = {"metric": "track-layer propagate+update/s", "value": res["network"]["value"],
            "unit": "track-layer/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (network: bf16 in, f32 accumulate)", "data": "synthetic",
            "config": {"workload": f"learned p2r seed: {n} p2r tracks x {NLAYER} layers, network "
                                   f"8-64-64-1 trained on {args.seed_train_samples} propagations",
                       "inputs_exceed_l2": True},
            "roofline": {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": alu_ach / alu_peak, "traffic": None, "kernel": "fit_seeded_kernel",
                         "flops_per_track_layer": seeded_flops,
                         "network_tensor_tflops": mlp_flops * tl / (ms / 1e3) / 1e12},
            "clocks": clk, "gpu_launches": args.steps,
            "plain_fit": res["straight_line"], "seeded_fit": res["network"],
            "crossing_start_fit": res["crossing"],
            "path_length_step_alone_4M_states": alone, "held_out_seed_error": seed_err,
            "training": {"samples": args.seed_train_samples, "epochs": args.seed_epochs,
                         "batch": 4096, "seconds": train_s, "final_loss": float(curve[-1])}}
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = len(os.sched_getaffinity(0))
        done, k, t0 = 0, 0, time.perf_counter()
        while k * 50000 < n and time.perf_counter() - t0 < 10.0:
            sub = ts.subset(np.arange(k * 50000, min(n, (k + 1) * 50000)))
            oracle.fit_set(sub, nthreads=cores)
            done += sub.n * NLAYER
            k += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": done / dt, "unit": "track-layer/s", "cores": cores,
                                "kind": "oracle", "sample": f"{done // NLAYER} of {n} tracks "
                                f"(exact FP64 path lengths, no seed), {dt:.1f} s"}
    return line


def bench_hostlink(args, world, rank, local):
    """The host link under the end-to-end path: 1-D page-locked copies
    (1.6 GB each way), and per mode the fused fit on host buffers through
    the staged copies (fit_propagate_update_host) and in place over the link
    (fit_propagate_update_mapped), against the same fit on device buffers."""
    import torch
    from paper_2409_09228_gb300 import fit

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    def t_ms(fn, reps=5):
        fn()
        torch.cuda.synchronize(dev)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    nb = 1_600_000_000
    h = torch.empty(nb, dtype=torch.uint8).pin_memory()
    d = torch.empty(nb, dtype=torch.uint8, device=dev)
    res = {"h2d_1d_GBs": nb / t_ms(lambda: d.copy_(h, non_blocking=True)) / 1e6,
           "d2h_1d_GBs": nb / t_ms(lambda: h.copy_(d, non_blocking=True)) / 1e6}
    del h, d
    sets = workload(rank)
    n = NEVT * NTRK
    ntrk = [NTRK] * NEVT
    f = fit.Fitter(fit.Geometry(sets[0].B, sets[0].surf), fit.Geometry(sets[1].B, sets[1].surf),
                   device=local)
    for m, name in ((0, "p2r"), (1, "p2z")):
        s = sets[m]
        arrs = (s.par0, s.cov0, s.q, s.hpos, s.hcov)
        dd = [torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in arrs]
        out_d = f.outputs(n, ld=n)
        hin = [torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for v in arrs]
        hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out_d.items()
                if v is not None}
        kw = dict(par_out=hout["par"], cov_out=hout["cov"], q_out=hout["q"], chi2=hout["chi2"],
                  status=hout["status"], stream=stream)
        # bytes the fit moves over the link: track state in and out, and the hit
        # components the update reads (p2z: x, y and their 3 covariance entries)
        hit_frac = HIT_BYTES[m] / 36.0
        nbytes = int(sum(t.numel() * t.element_size() for t in hin[:3] + list(hout.values())) +
                     hit_frac * sum(t.numel() * t.element_size() for t in hin[3:]))
        ms = {"device": t_ms(lambda: f.run(*dd, ntrk, [m] * NEVT, out=out_d, stream=stream)),
              "staged": t_ms(lambda: fit.fit_propagate_update_host(f.h, *hin, ntrk, [m] * NEVT, **kw)),
              "mapped": t_ms(lambda: fit.fit_propagate_update_mapped(f.h, *hin, ntrk, [m] * NEVT, **kw))}
        res[name] = {"ms": ms, "host_bytes": nbytes,
                     "mapped_GBs": nbytes / ms["mapped"] / 1e6, "staged_GBs": nbytes / ms["staged"] / 1e6}
        f.sync(stream)
    f.close()
    if rank != 0:
        return None
    return {"metric": "host-link bandwidth and end-to-end time per mode", "value": res["p2z"]["mapped_GBs"],
            "unit": "GB/s", "config": {"workload": f"{NEVT} events x {NTRK} tracks x {NLAYER} layers "
                                                   f"per mode, page-locked host buffers"},
            "hostlink": res}


SECONDARY = {"uneven": bench_uneven, "adjoint": bench_adjoint, "seed": bench_seed,
             "f64": bench_f64, "layout": bench_layout, "find": bench_find}


def secondary(args, world, rank, local) -> dict:
    """The other workloads at their own configurations, each timed with CUDA
    events in its own function (the lines `--workload W` prints), reduced to
    the figures that characterise them: run after the headline measurement,
    outside its timed region, without their CPU baselines."""
    import copy
    import torch
    res = {}
    for name, fn in SECONDARY.items():
        a = copy.copy(args)
        a.no_cpu_baseline = True
        a.steps, a.warmup = min(args.steps, 10), 3
        t0 = time.perf_counter()
        try:
            line = fn(a, world, rank, local)
        except Exception as e:  # a failing side workload must not cost the headline line
            res[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
            continue
        finally:
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        if line is None:
            continue
        keep = {k: line[k] for k in ("metric", "value", "unit", "ms_per_step", "dtype", "config",
                                     "roofline") if k in line}
        for k in ("per_segment_launches", "plan_default", "plan_tuned", "plain_fit", "seeded_fit",
                  "crossing_start_fit", "held_out_seed_error", "training", "layouts",
                  "p2r_layers_with_a_hit", "p2r_iterations_per_track_layer"):
            if k in line:
                keep[k] = line[k]
        keep["wall_s"] = time.perf_counter() - t0
        res[name] = keep
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the other workloads after the headline measurement")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--one-stream", action="store_true",
                    help="time the step with both modes on one stream (default: two streams)")
    ap.add_argument("--nevt", type=int, default=NEVT, help="events per mode (default 100)")
    ap.add_argument("--workload", default="uniform",
                    choices=["uniform", "uneven", "adjoint", "seed", "f64", "layout", "find",
                             "hostlink"],
                    help="uniform: 100 x 9600 x 20 per mode (the default); uneven: the batched "
                         "form on 2000 events of log-normal size and mixed modes")
    ap.add_argument("--uneven-events", type=int, default=2000)
    ap.add_argument("--adjoint-tracks", type=int, default=100000)
    ap.add_argument("--seed-tracks", type=int, default=1000000)
    ap.add_argument("--seed-train-samples", type=int, default=4000000)
    ap.add_argument("--seed-epochs", type=int, default=400)
    args = ap.parse_args()
    set_nevt(args.nevt)
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload != "uniform":
        fn = bench_hostlink if args.workload == "hostlink" else SECONDARY[args.workload]
        line = fn(args, world, rank, local)
        if line is not None:
            print(json.dumps(line))
        return

    import torch
    from paper_2409_09228_gb300 import fit

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    fit.load()
    sets = workload(rank)
    geoms = [fit.Geometry(s.B, s.surf) for s in sets]
    f = fit.Fitter(geoms[0], geoms[1], device=local)
    n = NEVT * NTRK
    ld = n
    up = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
    dev_in = [[up(a) for a in (s.par0, s.cov0, s.q, s.hpos, s.hcov)] for s in sets]
    outs = [f.outputs(n, ld=ld) for _ in sets]
    ntrk = [NTRK] * NEVT
    stream = torch.cuda.current_stream(dev)
    side = torch.cuda.Stream(dev)
    fork, join = torch.cuda.Event(), torch.cuda.Event()

    def step(events=None):
        # both modes on one stream, one after the other (each launch
        # bracketed by events: the per-kernel times of the roofline)
        for m in (0, 1):
            if events is not None:
                events[m][0].record(stream)
            f.run(*dev_in[m], ntrk, [m] * NEVT, out=outs[m], stream=stream)
            if events is not None:
                events[m][1].record(stream)

    def step_two_streams():
        # The p2r and p2z events are independent: p2z runs on a second stream,
        # so that its blocks take the SMs that p2r's last wave leaves idle;
        # the step ends when both have.
        fork.record(stream)
        side.wait_event(fork)
        f.run(*dev_in[0], ntrk, [0] * NEVT, out=outs[0], stream=stream)
        f.run(*dev_in[1], ntrk, [1] * NEVT, out=outs[1], stream=side)
        join.record(side)
        stream.wait_event(join)

    fp32_probe = measure_fp32(local)
    per = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(2)]
           for _ in range(args.steps)]
    t_begin, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # The clock record starts before the warm-up steps, so that the GPU comes
    # to the timed region from them (through one synchronize), not from an
    # idle pause, which cost the timed steps ~2 %.
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.warmup):
        step() if args.one_stream else step_two_streams()
    st = f.sync(stream)
    assert st["nonfinite"] == 0 and st["no_intersection"] == 0, st
    torch.cuda.synchronize(dev)
    barrier(world)
    t_begin.record(stream)
    for k in range(args.steps):
        step(per[k]) if args.one_stream else step_two_streams()
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    ms = t_begin.elapsed_time(t_end) / args.steps
    ms_one_stream = ms
    if not args.one_stream:
        # the per-kernel times, each kernel alone on the GPU: as many steps
        # again on one stream, inside the clock record
        s_begin, s_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s_begin.record(stream)
        for k in range(args.steps):
            step(per[k])
        s_end.record(stream)
        torch.cuda.synchronize(dev)
        ms_one_stream = s_begin.elapsed_time(s_end) / args.steps
    clk = clocks.stop()
    barrier(world)
    ms = max_over_ranks(world, ms)
    ms_one_stream = max_over_ranks(world, ms_one_stream)
    kernel_ms = [statistics.mean(per[k][m][0].elapsed_time(per[k][m][1]) for k in range(args.steps))
                 for m in (0, 1)]
    st = f.sync(stream)
    units_per_step = 2 * n * NLAYER
    value = world * units_per_step / (ms / 1e3)

    # iterations of the p2r path-length step per track-layer, counted by the kernel
    # (the counters hold both timed passes with two streams)
    passes = 1 if args.one_stream else 2
    it_per = st["iterations"] / max(1, passes * args.steps * n * NLAYER)
    flops = [flops_p2r(it_per), FLOPS_P2Z]
    mufu = [mufu_p2r(it_per), MUFU_P2Z]
    dom = int(np.argmax(kernel_ms))
    name = ["fit_fused_p2r", "fit_fused_p2z"][dom]
    peaks = load_peaks()
    sms = sm_count(local)
    alu_peak = fp32_peak_tflops(peaks["sm_max_mhz"], sms)
    tl = n * NLAYER
    bpls = [bytes_per_track_layer(NLAYER, m) for m in (0, 1)]
    bpl = bpls[dom]
    alu_ach = flops[dom] * tl / (kernel_ms[dom] / 1e3) / 1e12
    hbm_ach = bpl * tl / (kernel_ms[dom] / 1e3) / 1e9
    t_alu = flops[dom] * tl / (alu_peak * 1e12)
    t_hbm = bpl * tl / (peaks["hbm_gbs"] * 1e9)
    t_mufu = mufu[dom] * tl / (mufu_peak_tops(peaks["sm_max_mhz"], sms) * 1e12)
    traffic = profiled_traffic(name)
    if t_alu >= t_hbm:
        roof = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": alu_ach / alu_peak,
                "peak_source": f"derived: {sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                               f"{peaks['sm_max_mhz']:.0f} MHz (max SM clock, "
                               f"{'MEASURED_PEAKS.json' if peaks['source'] == 'measured' else 'nominal'})"}
    else:
        roof = {"bound": "hbm", "achieved": hbm_ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hbm_ach / peaks["hbm_gbs"], "peak_source": peaks["source"]}
    roof.update({"traffic": traffic, "kernel": name, "kernel_ms": kernel_ms[dom],
                 "flops_per_track_layer": flops[dom], "mufu_per_track_layer": mufu[dom],
                 "bytes_per_track_layer": bpl,
                 "hbm_frac": hbm_ach / peaks["hbm_gbs"], "alu_frac": alu_ach / alu_peak,
                 "t_roof_us": {"alu": t_alu * 1e6, "hbm": t_hbm * 1e6, "mufu": t_mufu * 1e6},
                 "kernel_ms_p2r_p2z": kernel_ms,
                 "frac_p2r_p2z": [max(flops[m] * tl / (alu_peak * 1e12),
                                      bpls[m] * tl / (peaks["hbm_gbs"] * 1e9)) /
                                  (kernel_ms[m] / 1e3) for m in (0, 1)],
                 "fp32_probe": fp32_probe})

    # End to end through the C ABI on host buffers: one fit_propagate_update_host
    # call per step copies both modes' tracks and hits (the p2r events, then the
    # p2z events, in one page-locked array set) through the library's staging,
    # fits them and copies the results back.
    pinned_in = [torch.from_numpy(np.ascontiguousarray(
        np.concatenate([getattr(s, k) for s in sets], axis=-1))).pin_memory()
        for k in ("par0", "cov0", "q", "hpos", "hcov")]
    pinned_out = {k: torch.empty(v.shape[:-1] + (2 * n,), dtype=v.dtype).pin_memory()
                  for k, v in outs[0].items() if v is not None}
    h2d = sum(t.numel() * t.element_size() for t in pinned_in)
    d2h = sum(t.numel() * t.element_size() for t in pinned_out.values())
    ntrk_both, mode_both = ntrk * 2, [0] * NEVT + [1] * NEVT

    def e2e_step():
        o = pinned_out
        fit.fit_propagate_update_host(f.h, *pinned_in, ntrk_both, mode_both, par_out=o["par"],
                                      cov_out=o["cov"], q_out=o["q"], chi2=o["chi2"],
                                      status=o["status"], stream=stream)

    def e2e_mapped_step():
        o = pinned_out
        fit.fit_propagate_update_mapped(f.h, *pinned_in, ntrk_both, mode_both, par_out=o["par"],
                                        cov_out=o["cov"], q_out=o["q"], chi2=o["chi2"],
                                        status=o["status"], stream=stream)

    def time_e2e(fn):
        fn()
        torch.cuda.synchronize(dev)
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return max_over_ranks(world, e0.elapsed_time(e1) / args.e2e_steps)

    e2e_ms = {"staged": float("nan"), "mapped": float("nan")}
    if args.e2e_steps > 0:
        e2e_ms["staged"] = time_e2e(e2e_step)
        e2e_ms["mapped"] = time_e2e(e2e_mapped_step)
    f.sync(stream)
    f.close()

    # The same p2r launch from the straight-line start (FIT_START_LINE), after
    # the timed region: what the closed-form crossing start saves.
    fl = fit.Fitter(fit.Geometry(sets[0].B, sets[0].surf, start=fit.FIT_START_LINE), None,
                    device=local)
    for _ in range(args.warmup):
        fl.run(*dev_in[0], ntrk, [0] * NEVT, out=outs[0], stream=stream)
    fl.sync(stream)
    l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0.record(stream)
    for _ in range(args.steps):
        fl.run(*dev_in[0], ntrk, [0] * NEVT, out=outs[0], stream=stream)
    l1.record(stream)
    torch.cuda.synchronize(dev)
    st_line = fl.sync(stream)
    fl.close()
    line_start = {"kernel_ms": max_over_ranks(world, l0.elapsed_time(l1) / args.steps),
                  "iterations_per_track_layer": st_line["iterations"] / (args.steps * n * NLAYER)}

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": "track-layer/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded generator, paper Sec. 3.1 smearing)",
            "config": config_dict(args), "roofline": roof, "clocks": clk,
            "e2e": {"value": world * units_per_step / (min(e2e_ms.values()) / 1e3),
                    "unit": "track-layer/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "path": min(e2e_ms, key=e2e_ms.get),
                    "paths": {"staged": "one fit_propagate_update_host call per step on "
                                        "page-locked host buffers holding both modes (chunked "
                                        "copies in, fit, copies out, three streams)",
                              "mapped": "one fit_propagate_update_mapped call per step: the "
                                        "fused kernels read the page-locked inputs and write the "
                                        "outputs over the host link, no staging copies"},
                    "ms_per_step": e2e_ms},
            "gpu_launches": 2 * args.steps,
            "step_streams": 1 if args.one_stream else 2, "ms_per_step_one_stream": ms_one_stream,
            "p2r_iterations_per_track_layer": it_per,
            "p2r_straight_line_start": line_start}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sets)
    if world == 1 and not args.no_secondary:
        line["secondary"] = secondary(args, world, rank, local)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
