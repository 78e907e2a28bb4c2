#!/usr/bin/env python3
"""Throughput benchmark of the synchronous NaSch step on the large road.

Workload: one ring of L = 2^31 cells holding N = 2^27 cars (density 1/16),
vmax = 5, p = 0.13, seed 1, Floyd start, T = 10^4 steps (the default run
times 10 benchmark steps of 1000 NaSch steps each = the whole T).  The
state (640 MiB agent, 2 GiB grid) is far larger than L2, so no flush is
needed between timed iterations.

Metric: vehicle-updates/s = N * NaSch steps / second (whole job, all ranks).
The JSON line also reports the fraction of the HBM roofline of the dominant
kernel, the end-to-end rate through the C ABI with host buffers, the other
layout's rate, and the oracle timed on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs its own replica road (road id =
rank): the road does not shard without a halo exchange, so N GPUs run N
independent replicas ("weak" scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2309_14311_gb300 import workloads as WL  # noqa: E402

STEPS_PER_BENCH_STEP = 1000
FALLBACK_HBM_GBS = 6800.0

# Algorithmic state bytes moved per unit by one fused launch (read + write):
# agent 4+1 bytes read and written per car, grid 1 byte read and written per cell.
AGENT_BYTES_PER_CAR = 10
GRID_BYTES_PER_CELL = 2


# --------------------------------------------------------------------------- helpers
def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_road_ids(world: int) -> list[int]:
    """Road id of each rank's replica: the Philox counter word that keeps the
    replicas' random draws independent."""
    return list(range(world))


def aggregate(units_per_rank: list[float], seconds_per_rank: list[float]) -> tuple[float, float]:
    """Whole-job rate: all units over the slowest rank's time."""
    t = max(seconds_per_rank)
    return sum(units_per_rank) / t, t


def reduce_over_ranks(value: float, op: str, device: str = "cuda") -> float:
    """max or sum of a scalar over the ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device_index)], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        with open(self.tmp.name) as f:
            rows = [[c.strip() for c in line.split(",")] for line in f if line.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The sources that define each measured kernel (a change to any of them
# invalidates its recorded traffic).
KERNEL_SOURCES = {
    "agent_tiled_k16": ("agent_kernels.cu", "tile_device.cuh", "nasch_device.cuh", "kernels.h"),
    "grid_k1": ("grid_kernels.cu", "tile_device.cuh", "nasch_device.cuh", "kernels.h"),
}


def source_tokens(text: str) -> str:
    """C/C++/CUDA source with its comments removed and every run of
    whitespace made one space: what a compiler sees, so that an edit of a
    comment or of the layout leaves it unchanged.  String and character
    literals are kept as they are."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":                              # literal: copy up to its closing quote
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):                # line comment
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):                # block comment
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2309_14311_gb300", "csrc")
    for fn in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, fn), encoding="utf-8") as f:
            h.update(source_tokens(f.read()).encode())
    return h.hexdigest()[:16]


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of the small profiling case (bench.py --profile; --set full,
# or the two DRAM counters alone),
# scaled to a launch of the large road by the units it processes (x4 cars for
# the agent kernel, x8 cells for the grid kernel; the traffic of these
# streaming kernels grows in proportion).  Keyed by the hash of the kernel's
# sources (comments and layout aside) when it was captured: a changed kernel
# reports null until it is captured again.
NCU_TRAFFIC: dict[str, dict] = {
    "agent_tiled_k16": {"source_hash": "73442a51b6bf5fae", "captured_bytes": 167842816 + 122001920,
                        "scale": 4, "bytes_per_launch": 4 * (167842816 + 122001920)},
    "grid_k1": {"source_hash": "2d862bad5c83bbfc", "captured_bytes": 268503040 + 219495680,
                "scale": 8, "bytes_per_launch": 8 * (268503040 + 219495680)},
}


def traffic_for(kernel: str):
    rec = NCU_TRAFFIC.get(kernel)
    if rec and rec.get("source_hash") == kernel_source_hash(kernel):
        return rec["bytes_per_launch"]
    return None


# --------------------------------------------------------------------------- oracle (CPU) arm
def time_oracle(spec: WL.RoadSpec, steps_per_sample: int, samples: int, warmup: int):
    """Oracle (OpenMP build) on the host cores: full ring, a bounded number of
    NaSch steps.  Returns (vehicle-updates/s, cores, seconds timed)."""
    import numpy as np

    # one thread per core, pinned (the OpenMP runtime reads these when the
    # oracle's OpenMP build is first loaded)
    os.environ.setdefault("OMP_PROC_BIND", "close")
    os.environ.setdefault("OMP_PLACES", "cores")
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    used = O.set_threads(cores)
    x = O.floyd_init(spec.L, spec.N, spec.seed, spec.road_id)
    v = np.zeros(spec.N, np.uint8)
    step = 0
    for _ in range(warmup):
        x, v, _, _ = O.agent_run(spec.L, x, v, spec.vmax, spec.p, spec.seed, spec.road_id, step, steps_per_sample,
                                 openmp=True)
        step += steps_per_sample
    times = []
    for _ in range(samples):
        t0 = time.perf_counter()
        x, v, _, _ = O.agent_run(spec.L, x, v, spec.vmax, spec.p, spec.seed, spec.road_id, step, steps_per_sample,
                                 openmp=True)
        times.append(time.perf_counter() - t0)
        step += steps_per_sample
    total = sum(times)
    return spec.N * steps_per_sample * samples / total, used, total, times


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def time_oracle_serial(spec: WL.RoadSpec, steps: int):
    """The serial oracle build on one core: `steps` NaSch steps of the full
    ring.  Returns (vehicle-updates/s, seconds)."""
    import numpy as np

    from oracle import oracle as O
    x = O.floyd_init(spec.L, spec.N, spec.seed, spec.road_id)
    v = np.zeros(spec.N, np.uint8)
    t0 = time.perf_counter()
    O.agent_run(spec.L, x, v, spec.vmax, spec.p, spec.seed, spec.road_id, 0, steps, openmp=False)
    sec = time.perf_counter() - t0
    return spec.N * steps / sec, sec


def workload_config(spec: WL.RoadSpec, world: int) -> dict:
    """The benchmark's workload, the same for both arms: the road, its
    replicas and the state's layout.  How many NaSch steps a benchmark step
    holds is a property of each arm's timing and goes in its `timing`."""
    return {"workload": spec.name, "L": spec.L, "N": spec.N, "vmax": spec.vmax, "p": spec.p, "seed": spec.seed,
            "road_ids": replica_road_ids(world), "layout": "agent", "parallelism": f"replicas{world}",
            "l2_flush": "not needed: agent state 640 MiB > 129 MB L2"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    spec = WL.LARGE_ROAD
    rate, cores, total, times = time_oracle(spec, args.ref_steps_per_step, args.steps, args.warmup)
    line = {
        "impl": "reference",
        "metric": "vehicle-updates/s",
        "value": rate,
        "unit": "vehicle-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": workload_config(spec, world),
        "timing": {"steps_per_bench_step": args.ref_steps_per_step,
                   "nasch_steps_timed": args.ref_steps_per_step * args.steps},
        "cpu_baseline": {"value": rate, "unit": "vehicle-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"full ring, {args.steps} x {args.ref_steps_per_step} NaSch steps "
                                   f"of the {spec.N}-car road (OpenMP oracle)", "cpu_model": cpu_model()},
        "e2e": {"value": rate, "unit": "vehicle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
# The agent step is bound by the SM's heavy integer-multiply pipe
# (fmaheavy), which runs Philox4x32-10's 32x32->64 products.  Per SM it
# takes 4 schedulers x 16 lanes = 64 lane-slots per clock; a 32x32->64
# product (IMAD.WIDE) occupies two slots, and so does a high half alone; a
# low half, an add or a move one (the ncu pipe counters fit these weights).
# Algorithmic work of one car-step: word 0 of Philox with counter (cell,
# step, road, 0) needs 13 wide products (rounds 1-7, less the product of the
# launch-constant road word in round 1 and of the step-constant word 0 in
# round 2, and round 8's word-0 product), 3 high halves (rounds 8, 9, 10)
# and 1 low half (round 9) = 26 + 6 + 1 = 33 lane-slots; the rules, the
# move and the statistics need none.
HEAVY_SLOTS_PER_CAR_STEP = 33
HEAVY_SLOTS_PER_SM_CLOCK = 64
# Algorithmic integer instructions of one car-step (issue view, kept beside
# it): Philox word 0 = 37 (two products and two 3-input xors per round, less
# the constant products and the last round's unused outputs), rules 1-4 with
# the statistics = 10.
ALU_OPS_PER_CAR_STEP = 47


def sm_clock_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except Exception:
        return 2070.0


def heavy_pipe_peak(props) -> tuple[float, str]:
    """Heavy-multiply-pipe ceiling in lane-slots per second: SMs x 64 slots
    per clock x the maximum SM clock."""
    mhz = sm_clock_mhz()
    return (props.multi_processor_count * HEAVY_SLOTS_PER_SM_CLOCK * mhz * 1e6,
            f"{props.multi_processor_count} SMs x {HEAVY_SLOTS_PER_SM_CLOCK} fmaheavy lane-slots per clock x "
            f"{mhz:.0f} MHz")


def issue_peak_ops(props) -> tuple[float, str]:
    """Integer issue ceiling: SMs x 4 schedulers x 32 lanes x max SM clock
    (one instruction per lane per clock)."""
    mhz = sm_clock_mhz()
    return props.multi_processor_count * 128 * mhz * 1e6, f"{props.multi_processor_count} SMs x 128 lanes x {mhz:.0f} MHz"


def run_ours(args):
    import numpy as np
    import torch

    from paper_2309_14311_gb300 import nasch as NS

    world, rank, local = dist_env()
    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    NS.load(build_if_missing=True)
    props = torch.cuda.get_device_properties(local)

    spec = WL.LARGE_ROAD
    road_id = replica_road_ids(world)[rank]
    layout = args.layout
    k = args.k or WL.LARGE_ROAD_K[layout]
    chunk = args.chunk
    stream = torch.cuda.Stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v: float) -> float:
        return reduce_over_ranks(v, "max")

    def sum_over_ranks(v: float) -> float:
        return reduce_over_ranks(v, "sum")

    def timed_device_run(road, nsteps_per_iter, iters, sampler=None):
        """CUDA events on the road's stream around `iters` calls of run()."""
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            start.record(stream)
            for _ in range(iters):
                road.run(nsteps_per_iter)
            end.record(stream)
            end.synchronize()
        torch.cuda.synchronize()
        barrier()
        return start.elapsed_time(end) / 1000.0

    # ---------------------------------------------------------------- main (device-resident) measurement
    road = NS.Road(spec.L, spec.N, spec.vmax, spec.p, spec.seed, road_id, layout=layout, k=k, stream=stream)
    info = road.info()
    for _ in range(args.warmup):
        road.run(chunk)
    road.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    secs = timed_device_run(road, chunk, args.steps, sampler)
    clocks = sampler.summary()
    t_max = max_over_ranks(secs)
    units = spec.N * chunk * args.steps
    total_units = sum_over_ranks(units)
    value = total_units / t_max
    launches_per_run = -(-chunk // info.k) if not info.ring_kernel else 1
    gpu_launches = launches_per_run * args.steps
    launch_s = secs / gpu_launches          # includes the two statistics memsets per run() call
    hbm_peak, hbm_kind = measured_peaks()
    kernel_name = f"{layout}_tiled_k{info.k}"
    car_steps_per_launch = spec.N * info.k
    if layout == "agent":
        heavy_peak, heavy_how = heavy_pipe_peak(props)
        achieved = HEAVY_SLOTS_PER_CAR_STEP * car_steps_per_launch / launch_s
        ops_peak, ops_how = issue_peak_ops(props)
        achieved_ops = ALU_OPS_PER_CAR_STEP * car_steps_per_launch / launch_s
        roofline = {"bound": "alu", "pipe": "fmaheavy", "achieved": achieved / 1e12, "peak": heavy_peak / 1e12,
                    "unit": "T fmaheavy lane-slots/s", "frac": achieved / heavy_peak,
                    "traffic": traffic_for(kernel_name), "kernel": kernel_name,
                    "peak_source": f"derived: {heavy_how} (a 32x32->64 product takes two slots)",
                    "algorithmic_slots_per_car_step": HEAVY_SLOTS_PER_CAR_STEP,
                    "car_steps_per_s_ceiling": heavy_peak / HEAVY_SLOTS_PER_CAR_STEP,
                    "issue_view": {"achieved_tops": achieved_ops / 1e12, "peak_tops": ops_peak / 1e12,
                                   "frac": achieved_ops / ops_peak, "ops_per_car_step": ALU_OPS_PER_CAR_STEP,
                                   "peak_source": f"derived: {ops_how}, one instruction per lane per clock"},
                    "algorithmic_bytes_per_launch": AGENT_BYTES_PER_CAR * spec.N,
                    "hbm_gbs": AGENT_BYTES_PER_CAR * spec.N / launch_s / 1e9, "launch_ms": launch_s * 1e3}
    else:
        alg = GRID_BYTES_PER_CELL * spec.L
        roofline = {"bound": "hbm", "achieved": alg / launch_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                    "frac": alg / launch_s / 1e9 / hbm_peak, "traffic": traffic_for(kernel_name),
                    "kernel": kernel_name, "peak_source": f"{hbm_kind} hbm_gbs",
                    "algorithmic_bytes_per_launch": alg, "launch_ms": launch_s * 1e3}
    philox_rate = NS.calibrate_philox(1 << 14)

    # ---------------------------------------------------------------- the HBM-bound form: grid at k = 1
    g1 = NS.Road(spec.L, spec.N, spec.vmax, spec.p, spec.seed, road_id, layout="grid", k=1, stream=stream)
    g1.run(20)
    g1.synchronize()
    # k1_steps launches of one step, back to back; the median of three such runs
    s1 = sorted(timed_device_run(g1, args.k1_steps, 1) for _ in range(3))[1]
    b1 = GRID_BYTES_PER_CELL * spec.L
    roofline_hbm = {"bound": "hbm", "kernel": "grid_k1", "achieved": b1 * args.k1_steps / s1 / 1e9,
                    "peak": hbm_peak, "unit": "GB/s", "frac": b1 * args.k1_steps / s1 / 1e9 / hbm_peak,
                    "traffic": traffic_for("grid_k1"), "peak_source": f"{hbm_kind} hbm_gbs",
                    "algorithmic_bytes_per_launch": b1, "launch_ms": s1 / args.k1_steps * 1e3,
                    "vehicle_updates_per_s": spec.N * args.k1_steps / s1,
                    "cell_updates_per_s": spec.L * args.k1_steps / s1}
    gk = WL.LARGE_ROAD_K["grid"]
    g1.close()
    gr = NS.Road(spec.L, spec.N, spec.vmax, spec.p, spec.seed, road_id, layout="grid", k=gk, stream=stream)
    gr.run(gk)
    gr.synchronize()
    gsteps = max(gk, (args.other_steps // gk) * gk)
    sg = timed_device_run(gr, gsteps, 1)
    grid_res = {"layout": "grid", "k": gk, "vehicle_updates_per_s": spec.N * gsteps / sg,
                "cell_updates_per_s": spec.L * gsteps / sg, "steps_timed": gsteps}
    gr.close()

    # ---------------------------------------------------------------- end to end through the C ABI, host buffers
    x_host = torch.empty(spec.N, dtype=torch.int32, pin_memory=True).numpy()
    v_host = torch.empty(spec.N, dtype=torch.uint8, pin_memory=True).numpy()
    sv_host = np.zeros(chunk, np.uint64)
    cr_host = np.zeros(chunk, np.uint64)
    road.read_state(x_host, v_host)
    step0 = road.step
    e2e_iters = max(1, args.e2e_steps)
    lib = NS.load()
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_iters):
        road.set_state(x_host, v_host, step0 + i * chunk)        # host -> device
        road.run(chunk)
        road.read_state(x_host, v_host)                          # device -> host
        NS._check(lib.nasch_stats(road.handle, step0 + i * chunk, chunk, NS._ptr(sv_host), NS._ptr(cr_host)))
    e2e_secs = max_over_ranks(time.perf_counter() - t0)
    barrier()
    e2e_units = sum_over_ranks(spec.N * chunk * e2e_iters)
    road.close()

    # ---------------------------------------------------------------- batched vs plain, and served
    batch_res = run_batch_vs_plain(args, NS, stream, torch) if not args.no_batch else None
    serve_res = run_served(args, NS, batch_res) if (not args.no_serve and batch_res) else None
    saturated = (run_serve_vs_batch(args, NS, stream, WL.request_stream()[: args.serve_requests])
                 if not args.no_serve else None)
    ensemble = None
    if not args.no_ensemble:
        ensemble = ensemble_vs_plain(NS, stream, torch, WL.uneven_ensemble(), args.plain_roads)
        ensemble["sample"] = (f"the whole seed-7 ensemble batched; {args.plain_roads} of its roads (seed 7) run "
                              f"one per launch")

    # ---------------------------------------------------------------- oracle on the host cores (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, total, _ = time_oracle(spec, args.cpu_steps, 1, 0)
        srate, ssec = time_oracle_serial(spec, 1)
        cpu = {"value": rate, "unit": "vehicle-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"full ring of {spec.N} cars, {args.cpu_steps} NaSch steps, OpenMP oracle, "
                         f"{total:.1f} s",
               "cpu_model": cpu_model(), "threads": "one per core, pinned (OMP_PROC_BIND=close, OMP_PLACES=cores)",
               "serial_1core": {"value": srate, "unit": "vehicle-updates/s", "cores": 1,
                                "sample": f"full ring of {spec.N} cars, 1 NaSch step, serial oracle, {ssec:.1f} s"}}

    if rank == 0:
        line = {
            "metric": "vehicle-updates/s",
            "value": value,
            "unit": "vehicle-updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1000.0 * t_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "int32",
            "data": "synthetic",
            "config": dict(workload_config(spec, world), layout=layout),
            "timing": {"k": info.k, "steps_per_bench_step": chunk, "nasch_steps_timed": chunk * args.steps},
            "roofline": roofline,
            "roofline_hbm": roofline_hbm,
            "philox_ceiling": {"draws_per_s": philox_rate, "frac": value / world / philox_rate,
                               "note": "bare rule-3 draws per second (nasch_calibrate_philox); one per car-step"},
            "cell_updates_per_s": value * spec.L / spec.N,
            "grid_layout": grid_res,
            "e2e": {"value": e2e_units / e2e_secs, "unit": "vehicle-updates/s",
                    "h2d_bytes_per_step": spec.N * 5, "d2h_bytes_per_step": spec.N * 5 + chunk * 16},
            "batched_vs_plain": batch_res,
            "served": serve_res,
            "served_saturated_vs_batched": saturated,
            "ensemble_4096": ensemble,
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch_vs_plain(args, NS, stream, torch):
    """A seeded sample of the uneven ensemble (L log-uniform 1e3..1e7, T
    log-uniform 1e3..1e5): all roads in one batched job vs the same roads one
    after another through the single-road API (plain per-road launches).
    GPU time only (start states excluded on both sides)."""
    import numpy as np
    rows = WL.uneven_ensemble()
    rng = np.random.default_rng(2309)
    idx = sorted(rng.choice(len(rows), args.batch_roads, replace=False).tolist())
    roads = [WL.road_params(rows[i]) for i in idx]
    steps = [rows[i]["T"] for i in idx]
    work = sum(r["N"] * t for r, t in zip(roads, steps))
    with NS.Batch(roads, steps, stream=stream) as b:
        b.wait()
        inf = b.info()
        batched_s = inf.run_seconds
    plain_s = 0.0
    launches = 0
    for r, t in zip(roads, steps):
        with NS.Road(r["L"], r["N"], r["vmax"], r["p"], r["seed"], r["road_id"], stream=stream) as road:
            ri = road.info()
            road.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            road.run(t)
            e.record(stream)
            e.synchronize()
            plain_s += a.elapsed_time(e) / 1e3
            launches += 1 if ri.ring_kernel else -(-t // ri.k)
    return {"roads": len(roads), "sample": f"{len(roads)} roads drawn (seed 2309) from the seed-7 ensemble table",
            "vehicle_updates": work, "batched_vehicle_updates_per_s": work / batched_s,
            "plain_vehicle_updates_per_s": work / plain_s, "speedup": plain_s / batched_s,
            "batched_launches": int(inf.super_steps), "plain_launches": launches,
            "batched_seconds": batched_s, "plain_seconds": plain_s}


def run_served(args, NS, batch_res):
    """The first requests of the seed-11 stream served by the continuous-batching
    loop at an offered load of `serve_load` x the batched capacity."""
    from paper_2309_14311_gb300 import serve as SV
    rows = WL.request_stream()[: args.serve_requests]
    mean_work = sum(r["N"] * r["T"] for r in rows) / len(rows)
    capacity = batch_res["batched_vehicle_updates_per_s"] / mean_work     # requests per second
    rate = args.serve_load * capacity
    out = SV.run_poisson(rows, rate=rate, memory_budget=args.serve_budget_gb << 30,
                         steps_per_tick=args.serve_steps_per_tick, time_limit_s=args.serve_time_limit)
    out["offered_load"] = args.serve_load
    out["steps_per_tick"] = args.serve_steps_per_tick
    out["budget_bytes"] = args.serve_budget_gb << 30
    return out


def ensemble_vs_plain(NS, stream, torch, rows, plain_roads, seed=7):
    """Roads of the uneven ensemble in one batched job, and a seeded subset of
    `plain_roads` of them one after another through the single-road API
    (plain per-road launches); GPU time only on both sides (start states
    excluded)."""
    roads = [WL.road_params(r) for r in rows]
    steps = [r["T"] for r in rows]
    work = sum(r["N"] * r["T"] for r in rows)
    t0 = time.perf_counter()
    with NS.Batch(roads, steps, stream=stream) as b:
        b.wait()
        inf = b.info()
        layouts = [b.layout(i) for i in range(len(rows))]
    wall = time.perf_counter() - t0
    out = dict(roads=len(rows), vehicle_updates=work, batched_gpu_seconds=inf.run_seconds, batched_wall_seconds=wall,
               batched_vehicle_updates_per_s=work / inf.run_seconds, super_steps=int(inf.super_steps),
               graphs=int(inf.graphs), device_bytes=int(inf.device_bytes),
               agent_roads=sum(1 for x in layouts if x == NS.LAYOUT_AGENT))
    if plain_roads <= 0:
        return out
    out.update(plain_launches(NS, stream, torch, rows, plain_roads, seed))
    out["speedup"] = (work / inf.run_seconds) / out["plain_vehicle_updates_per_s"]
    return out


def plain_launches(NS, stream, torch, rows, plain_roads, seed):
    """A seeded subset of `plain_roads` of the roads run one after another
    through the single-road API (one road per launch), GPU time only."""
    import numpy as np
    sub = list(range(len(rows)))
    if plain_roads < len(rows):
        rng = np.random.default_rng(seed)
        sub = sorted(rng.choice(len(rows), plain_roads, replace=False).tolist())
    pwork = sum(rows[i]["N"] * rows[i]["T"] for i in sub)
    plain = 0.0
    for i in sub:
        r = rows[i]
        with NS.Road(r["L"], r["N"], r["vmax"], r["p"], r["seed"], r["road_id"], stream=stream) as road:
            road.synchronize()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            road.run(r["T"])
            e.record(stream)
            e.synchronize()
            plain += a.elapsed_time(e) / 1e3
    return dict(plain_roads=len(sub), plain_vehicle_updates=pwork, plain_gpu_seconds=plain,
                plain_vehicle_updates_per_s=pwork / plain)


def run_serve_vs_batch(args, NS, stream, rows):
    """The same requests batched (one nasch_submit job) and served all at
    once (saturated continuous batching): GPU rates of both and the served
    fraction of the batched rate, with the server's GPU-busy fraction."""
    from paper_2309_14311_gb300 import serve as SV
    roads = [WL.road_params(r) for r in rows]
    steps = [r["T"] for r in rows]
    work = sum(r["N"] * r["T"] for r in rows)
    t0 = time.perf_counter()
    with NS.Batch(roads, steps, stream=stream) as b:
        b.wait()
        batched_s = b.info().run_seconds
    batched_wall = time.perf_counter() - t0          # start states included, as for the served requests
    out = SV.run_poisson(rows, rate=float("inf"), memory_budget=args.serve_budget_gb << 30,
                         steps_per_tick=args.serve_steps_per_tick, time_limit_s=args.serve_time_limit,
                         stream_series=True)
    served = out["vehicle_updates_per_s"]
    import torch
    plain = plain_launches(NS, stream, torch, rows, min(64, len(rows)), seed=11)
    return {"requests": len(rows), "vehicle_updates": work, "batched_vehicle_updates_per_s": work / batched_s,
            "plain_vehicle_updates_per_s": plain["plain_vehicle_updates_per_s"],
            "plain_sample": f"{plain['plain_roads']} of the requests (seed 11) run one road per launch",
            "served_over_plain": served / plain["plain_vehicle_updates_per_s"],
            "batched_with_start_states_vehicle_updates_per_s": work / batched_wall,
            "served_vehicle_updates_per_s": served, "served_over_batched": served / (work / batched_s),
            "served_gpu_busy_fraction": out["gpu_busy_fraction"], "served_span_s": out["span_s"],
            "ticks": out["ticks"], "streamed_steps": out["streamed_steps"],
            "all_steps": sum(steps), "sample": f"the first {len(rows)} requests of the seed-11 stream, all queued at "
                                               f"once"}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


# --------------------------------------------------------------------------- other workloads (one JSON line each)
def run_workload(args):
    """The batched and served configurations, measured on their own:

    ensemble             the seed-7 uneven ensemble (4096 roads, or the first
                         --roads of a seeded sample), batched in one job vs
                         plain per-road launches (--plain-roads of them);
    fundamental-diagram  the density sweep: 64 densities x p in {0, 0.13, 0.25,
                         0.5} x --replicas replicas, L = --fd-L, T = 12000 with
                         the first 2000 steps discarded; time-averaged flux and
                         velocity per (density, p), and for p = 0 the
                         deterministic steady state min(vmax rho, 1 - rho);
    serve                the seed-11 request stream (first --serve-requests),
                         Poisson arrivals at --serve-load x capacity, 40 GB
                         budget; p50/p99 latency and aggregate rate;
    decomposed           a 2^30-cell ring split over 1, 2 and 4 cell ranges
                         (every rank on this GPU, one after another):
                         the segment kernel's rate per rank and the halo
                         bytes of an exchange;
    serve-vs-batch       the first --serve-requests requests batched in one
                         job and served all at once (series streamed back):
                         the served rate as a fraction of the batched one;
    snapshots            output while running: a 2^28-cell road (2^24 cars)
                         run for --other-steps steps with no output, with
                         snapshots of its cells every 50 and every 10 steps
                         (pinned host ring of 4 slots), and with a 4096-pixel
                         space-time raster row every step; the slowdown of
                         each against no output;
    open-road            the large road opened (entry alpha = 0.5 before cell
                         0, exit beta = 0.5 after cell L-1; grid layout, one
                         step per launch): rates over --other-steps steps
                         and the fraction of the measured HBM copy bandwidth
                         (2 B per cell-step);
    k-sweep              the large road (2^31 cells, 2^27 cars) in each
                         layout at each fusion depth k of --sweep-k: rates
                         over --other-steps steps after 2k warm-up steps."""
    import numpy as np
    import torch

    from paper_2309_14311_gb300 import nasch as NS
    torch.cuda.set_device(0)
    NS.load(build_if_missing=True)
    stream = torch.cuda.Stream()
    out = {"workload": args.workload}
    if args.workload == "open-road":
        spec = WL.LARGE_ROAD
        steps = max(args.other_steps, 10)
        with NS.Road(spec.L, spec.N, spec.vmax, spec.p, spec.seed, spec.road_id, layout="grid", open=(0.5, 0.5),
                     stream=stream) as r:
            r.run(5)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r.run(steps)
            b.record(stream)
            b.synchronize()
            sec = a.elapsed_time(b) / 1e3
            cells = r.read_grid()
            cars_now = int((cells >= 0).sum())
        hbm_peak, hbm_kind = measured_peaks()
        gbs = 2.0 * spec.L * steps / sec / 1e9
        out.update(L=spec.L, N_start=spec.N, cars_after=cars_now, alpha=0.5, beta=0.5, steps=steps,
                   cell_updates_per_s=spec.L * steps / sec, launch_ms=sec / steps * 1e3,
                   roofline_hbm={"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": gbs / hbm_peak, "peak_source": f"{hbm_kind} hbm_gbs"})
    elif args.workload == "snapshots":
        L, N = 1 << 28, 1 << 24
        steps = max(args.other_steps, 100) // 100 * 100
        pinned = torch.empty((4, L), dtype=torch.int8, pin_memory=True)
        snaps = pinned.numpy()
        rows = np.zeros((steps, 4096), np.uint8)
        rows_out = []
        for layout, k in (("agent", 16), ("grid", 1)):
            with NS.Road(L, N, 5, 0.13, 1, 0, layout=layout, k=k, stream=stream) as r:
                r.run_output(2 * k, k, snaps, rows[:2])   # warm-up, and the staging buffers made
                res = {}
                for name, per, sn, rw in (("off", 0, None, None), ("snap_every_50", 50, snaps, None),
                                          ("snap_every_10", 10, snaps, None), ("raster_every_1", 1, None, rows)):
                    t0 = time.perf_counter()
                    r.run_output(steps, per, sn, rw)
                    sec = time.perf_counter() - t0
                    res[name] = {"vehicle_updates_per_s": N * steps / sec, "seconds": sec}
                base = res["off"]["seconds"]
                for v in res.values():
                    v["slowdown"] = v["seconds"] / base
                rows_out.append({"layout": layout, "k": k, "steps": steps, "snapshot_bytes": L, **res})
        out.update(L=L, N=N, rows=rows_out)
    elif args.workload == "k-sweep":
        s = WL.LARGE_ROAD
        rows = []
        for layout in ("agent", "grid"):
            for k in [int(t) for t in args.sweep_k.split(",")]:
                steps = max(args.other_steps // k, 1) * k
                with NS.Road(s.L, s.N, s.vmax, s.p, s.seed, s.road_id, layout=layout, k=k, stream=stream) as r:
                    r.run(2 * k)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    r.run(steps)
                    b.record(stream)
                    b.synchronize()
                    sec = a.elapsed_time(b) / 1e3
                    k_used = r.info().k
                rows.append({"layout": layout, "k": k, "k_used": int(k_used), "steps": steps,
                             "vehicle_updates_per_s": s.N * steps / sec, "cell_updates_per_s": s.L * steps / sec,
                             "algorithmic_gbs": (10 * s.N if layout == "agent" else 2 * s.L) * steps / k_used / sec
                             / 1e9})
        out.update(L=s.L, N=s.N, vmax=s.vmax, p=s.p, rows=rows)
    elif args.workload == "ensemble":
        rows = WL.uneven_ensemble()
        if args.roads < len(rows):
            rng = np.random.default_rng(2309)
            rows = [rows[i] for i in sorted(rng.choice(len(rows), args.roads, replace=False).tolist())]
        if args.autotune:
            from paper_2309_14311_gb300 import autotune as AT
            untuned = ensemble_vs_plain(NS, stream, torch, rows, 0)
            t0 = time.perf_counter()
            AT.load_or_tune_buckets()
            out["autotune_seconds"] = time.perf_counter() - t0
            out["untuned_batched_vehicle_updates_per_s"] = untuned["batched_vehicle_updates_per_s"]
        out.update(ensemble_vs_plain(NS, stream, torch, rows, args.plain_roads))
        if args.autotune:
            out["tuned_over_untuned"] = out["batched_vehicle_updates_per_s"] / out["untuned_batched_vehicle_updates_per_s"]
            NS.set_tuning_table([])
    elif args.workload == "fundamental-diagram":
        from paper_2309_14311_gb300 import fundamental as FD
        roads = WL.fundamental_diagram_roads(replicas=args.replicas, L=args.fd_L, vmax=args.fd_vmax)
        T = WL.FD_T
        window = T - WL.FD_WARMUP
        t0 = time.perf_counter()
        with NS.Batch(roads, [T] * len(roads), stream=stream) as b:
            b.wait()
            inf = b.info()
            sums = [FD.ReplicaSum(r["L"], r["N"], r["p"], r["vmax"], b.stats_sum(i, WL.FD_WARMUP, window)[0], window)
                    for i, r in enumerate(roads)]
        wall = time.perf_counter() - t0
        rows = FD.fd_table(sums)
        work = sum(r["N"] for r in roads) * T
        out.update(roads=len(roads), L=args.fd_L, T=T, warmup=WL.FD_WARMUP, vmax=args.fd_vmax,
                   vehicle_updates=work, batched_gpu_seconds=inf.run_seconds, wall_seconds=wall,
                   vehicle_updates_per_s=work / inf.run_seconds, **FD.summary(rows), table=rows)
    elif args.workload == "decomposed":
        # one ring split over `world` cell ranges (the multi-GPU domain
        # decomposition), every rank's buffer on this GPU and the ranks run
        # one after another; per-rank segment-kernel time by CUDA events, the
        # halo exchange as device copies between the buffers
        from paper_2309_14311_gb300 import decomp as DC
        L, N, vmax, p, k = 1 << 30, 1 << 26, 5, 0.13, 8
        steps = max(args.other_steps // k, 2) * k
        x0 = NS.floyd_init(L, N, 1, 0)
        rows_out = []
        for world in (1, 2, 4):
            segs = DC.segments(L, world, k, vmax)
            bufs = []
            for sg in segs:
                b = torch.full((sg.W,), -1, dtype=torch.int8, device="cuda")
                j = (x0.astype(np.int64) - sg.a) % L
                b[torch.from_numpy(sg.H + j[j < sg.owned]).cuda()] = 0
                bufs.append(b)
            outs = [b.clone() for b in bufs]
            kernel_s = [0.0] * world
            base_step = DC.library_step(L, vmax, p, 1, 0, stream=torch.cuda.current_stream())

            def timed(seg, bi, bo, kk, s0, rank):
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                res = base_step(seg, bi, bo, kk, s0, rank)
                e.record()
                e.synchronize()
                kernel_s[rank] += a.elapsed_time(e) / 1e3
                return res

            DC.run_local(segs, bufs, 2 * k, base_step, spare=outs)            # warm-up
            torch.cuda.synchronize()
            kernel_s = [0.0] * world
            t0 = time.perf_counter()
            bufs2, _ = DC.run_local(segs, bufs, steps, timed, step0=2 * k, spare=outs)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            rows_out.append({"world": world, "steps": steps, "halo_cells": segs[0].H,
                             "halo_bytes_per_rank_per_launch": 2 * segs[0].H,
                             "segment_kernel_seconds_per_rank": kernel_s,
                             "cell_updates_per_s_per_rank_kernel": [sg.owned * steps / t for sg, t in zip(segs, kernel_s)],
                             "cell_updates_per_s_one_gpu_all_ranks": L * steps / wall})
        out.update(L=L, N=N, vmax=vmax, p=p, k=k, rows=rows_out,
                   note="ranks run one after another on one GPU; a rank's kernel rate is what one GPU per rank "
                        "would run at, before its halo exchange")
    elif args.workload == "serve-vs-batch":
        rows = WL.request_stream()[: args.serve_requests]
        out.update(run_serve_vs_batch(args, NS, stream, rows))
    elif args.workload == "serve":
        from paper_2309_14311_gb300 import serve as SV
        rows = WL.request_stream()[: args.serve_requests]
        mean_work = sum(r["N"] * r["T"] for r in rows) / len(rows)
        cap = args.serve_capacity or 3.5e11
        rate = args.serve_load * cap / mean_work
        res = SV.run_poisson(rows, rate=rate, memory_budget=args.serve_budget_gb << 30,
                             steps_per_tick=args.serve_steps_per_tick, time_limit_s=args.serve_time_limit)
        out.update(res, assumed_capacity_vehicle_updates_per_s=cap, offered_load=args.serve_load,
                   steps_per_tick=args.serve_steps_per_tick)
    print(json.dumps(out), flush=True)
    return 0


def run_profile_case(args):
    """A small case of one kernel for ncu captures: inputs larger than L2 but a
    few hundred MiB on the device; `--profile-launches` launches after two
    warm-up launches.  Prints nothing but a one-line summary."""
    import torch

    from paper_2309_14311_gb300 import nasch as NS
    torch.cuda.set_device(0)
    NS.load(build_if_missing=True)
    layout = args.profile
    k = args.k or WL.LARGE_ROAD_K[layout]
    # density 1/16 like the large road; agent 2^25 cars (160 MiB of state),
    # grid 2^28 cells (256 MiB)
    L, N = (2**29, 2**25) if layout == "agent" else (2**28, 2**24)
    road = NS.Road(L, N, 5, 0.13, 1, 0, layout=layout, k=k)
    road.run(2 * k)
    road.run(args.profile_launches * k)
    road.synchronize()
    print(f"profile case {layout} k={k} L={L} N={N} launches={2 + args.profile_launches}")
    road.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10, help="timed benchmark steps (1000 NaSch steps each)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--layout", choices=["agent", "grid"], default="agent")
    ap.add_argument("--k", type=int, default=0, help="fused steps per launch (0: tuned default)")
    ap.add_argument("--chunk", type=int, default=STEPS_PER_BENCH_STEP, help="NaSch steps per benchmark step")
    ap.add_argument("--other-steps", type=int, default=400)
    ap.add_argument("--k1-steps", type=int, default=100)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-roads", type=int, default=64)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the whole-ensemble batched-vs-plain leg")
    ap.add_argument("--autotune", action="store_true", help="ensemble workload: also per-road tuned")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-budget-gb", type=int, default=40)
    ap.add_argument("--serve-time-limit", type=float, default=120.0)
    ap.add_argument("--serve-steps-per-tick", type=int, default=8, help="super-step launches per scheduling round")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--ref-steps-per-step", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["large-road", "ensemble", "fundamental-diagram", "serve", "serve-vs-batch",
                                           "k-sweep", "snapshots", "open-road", "decomposed"],
                    default="large-road", help="large-road is the benchmark line; the others print their own line")
    ap.add_argument("--sweep-k", default="1,2,4,8,16,32", help="fusion depths of the k-sweep workload")
    ap.add_argument("--roads", type=int, default=4096)
    ap.add_argument("--plain-roads", type=int, default=256)
    ap.add_argument("--replicas", type=int, default=128)
    ap.add_argument("--fd-L", type=int, default=10**6)
    ap.add_argument("--fd-vmax", type=int, default=5, help="vmax of the fundamental-diagram roads (1: exact flux known)")
    ap.add_argument("--serve-capacity", type=float, default=0.0,
                    help="vehicle-updates/s the offered load is scaled to (0: 3.5e11)")
    ap.add_argument("--profile", choices=["agent", "grid"], default=None,
                    help="run the small ncu profiling case of one layout and exit")
    ap.add_argument("--profile-launches", type=int, default=3)
    args = ap.parse_args(argv)
    if args.profile:
        return run_profile_case(args)
    if args.workload != "large-road":
        return run_workload(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
