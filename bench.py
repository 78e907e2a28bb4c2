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


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2309_14311_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


# DRAM traffic per launch from an ncu capture of the dominant kernel, keyed by
# the kernel source hash it was taken on (None until a capture exists).
NCU_TRAFFIC: dict[str, dict] = {}


def traffic_for(kernel: str):
    rec = NCU_TRAFFIC.get(kernel)
    if rec and rec.get("source_hash") == kernel_source_hash():
        return rec["bytes_per_launch"]
    return None


# --------------------------------------------------------------------------- oracle (CPU) arm
def time_oracle(spec: WL.RoadSpec, steps_per_sample: int, samples: int, warmup: int):
    """Oracle (OpenMP build) on the host cores: full ring, a bounded number of
    NaSch steps.  Returns (vehicle-updates/s, cores, seconds timed)."""
    import numpy as np

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
        "config": {"workload": spec.name, "L": spec.L, "N": spec.N, "vmax": spec.vmax, "p": spec.p,
                   "seed": spec.seed, "layout": "agent", "steps_per_bench_step": args.ref_steps_per_step,
                   "l2_flush": "not needed: state 640 MiB > 129 MB L2"},
        "cpu_baseline": {"value": rate, "unit": "vehicle-updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"full ring, {args.steps} x {args.ref_steps_per_step} NaSch steps "
                                   f"of the {spec.N}-car road (OpenMP oracle)"},
        "e2e": {"value": rate, "unit": "vehicle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm
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

    result = {}
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
    launch_s = secs / gpu_launches
    if layout == "agent":
        alg_bytes = AGENT_BYTES_PER_CAR * spec.N
    else:
        alg_bytes = GRID_BYTES_PER_CELL * spec.L
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / launch_s / 1e9
    kernel_name = f"{layout}_tiled_k{info.k}"

    # ---------------------------------------------------------------- other layout, same road (context)
    other = "grid" if layout == "agent" else "agent"
    other_k = WL.LARGE_ROAD_K[other]
    other_road = NS.Road(spec.L, spec.N, spec.vmax, spec.p, spec.seed, road_id, layout=other, k=other_k,
                         stream=stream)
    other_steps = max(other_k, (args.other_steps // other_k) * other_k)
    other_road.run(other_steps)
    other_road.synchronize()
    o_secs = timed_device_run(other_road, other_steps, 1)
    o_launch_s = o_secs / (-(-other_steps // other_k))
    o_bytes = AGENT_BYTES_PER_CAR * spec.N if other == "agent" else GRID_BYTES_PER_CELL * spec.L
    other_res = {"layout": other, "k": other_k, "vehicle_updates_per_s": spec.N * other_steps / o_secs,
                 "cell_updates_per_s": spec.L * other_steps / o_secs,
                 "hbm_gbs": o_bytes / o_launch_s / 1e9, "hbm_frac": o_bytes / o_launch_s / 1e9 / peak,
                 "steps_timed": other_steps}
    other_road.close()

    # k = 1 form of each layout: the HBM-bound configuration of the step
    k1 = {}
    for lay in ("agent", "grid"):
        r1 = NS.Road(spec.L, spec.N, spec.vmax, spec.p, spec.seed, road_id, layout=lay, k=1, stream=stream)
        r1.run(5)
        r1.synchronize()
        s1 = timed_device_run(r1, 1, args.k1_steps)
        b1 = AGENT_BYTES_PER_CAR * spec.N if lay == "agent" else GRID_BYTES_PER_CELL * spec.L
        k1[lay] = {"k": 1, "vehicle_updates_per_s": spec.N * args.k1_steps / s1,
                   "hbm_gbs": b1 * args.k1_steps / s1 / 1e9, "hbm_frac": b1 * args.k1_steps / s1 / 1e9 / peak}
        r1.close()

    # ---------------------------------------------------------------- end to end through the C ABI, host buffers
    x_host = torch.empty(spec.N, dtype=torch.int32, pin_memory=True).numpy()
    v_host = torch.empty(spec.N, dtype=torch.uint8, pin_memory=True).numpy()
    sv_host = np.zeros(chunk, np.uint64)
    cr_host = np.zeros(chunk, np.uint64)
    road.read_state(x_host, v_host)
    step0 = road.step
    e2e_iters = max(1, args.e2e_steps)
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_iters):
        road.set_state(x_host, v_host, step0 + i * chunk)        # host -> device
        road.run(chunk)
        road.read_state(x_host, v_host)                          # device -> host
        lib = NS.load()
        NS._check(lib.nasch_stats(road.handle, step0 + i * chunk, chunk, NS._ptr(sv_host), NS._ptr(cr_host)))
    e2e_secs = max_over_ranks(time.perf_counter() - t0)
    barrier()
    e2e_units = sum_over_ranks(spec.N * chunk * e2e_iters)
    road.close()

    # ---------------------------------------------------------------- oracle on the host cores (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, total, _ = time_oracle(spec, args.cpu_steps, 1, 0)
        cpu = {"value": rate, "unit": "vehicle-updates/s", "cores": cores, "kind": "oracle",
               "sample": f"full ring of {spec.N} cars, {args.cpu_steps} NaSch steps, OpenMP oracle, "
                         f"{total:.1f} s"}

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
            "config": {"workload": spec.name, "L": spec.L, "N": spec.N, "vmax": spec.vmax, "p": spec.p,
                       "seed": spec.seed, "road_ids": replica_road_ids(world), "layout": layout, "k": info.k,
                       "steps_per_bench_step": chunk, "nasch_steps_timed": chunk * args.steps,
                       "parallelism": f"replicas{world}",
                       "l2_flush": "not needed: state 640 MiB (agent) / 4 GiB (grid) > 129 MB L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic_for(kernel_name),
                         "kernel": kernel_name, "peak_source": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "launch_ms": launch_s * 1e3},
            "cell_updates_per_s": value * spec.L / spec.N,
            "other_layout": other_res,
            "k1": k1,
            "e2e": {"value": e2e_units / e2e_secs, "unit": "vehicle-updates/s",
                    "h2d_bytes_per_step": spec.N * 5, "d2h_bytes_per_step": spec.N * 5 + chunk * 16},
            "gpu_launches": gpu_launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


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
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--ref-steps-per-step", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", choices=["agent", "grid"], default=None,
                    help="run the small ncu profiling case of one layout and exit")
    ap.add_argument("--profile-launches", type=int, default=3)
    args = ap.parse_args(argv)
    if args.profile:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
