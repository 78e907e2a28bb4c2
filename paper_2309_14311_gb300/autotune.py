"""Autotuner for the automatic launch choices.

Three choices are tuned by timing the library's own kernels through the C
ABI on this GPU:

* fusion depth k of tiled agent roads and of tiled grid roads: the k with the
  highest vehicle-updates/s on a representative road of each layout;
* rho*, the density below which AUTO picks the agent layout: for each
  density of a grid of densities the agent and grid layouts are timed (each
  at its tuned k) and rho* is put where the faster layout changes.

Results go to nasch_set_tuning() and to a JSON cache keyed by the GPU name
and the library build, so later processes reuse them without re-timing.

Per-road tuning of batches and servers (tune_buckets): roads are put in
buckets by L (decades), density (three bands) and vmax; for each bucket the
layout, the fusion depth k and the grid tile (warp-tiles or block-wide
spans) that ran a batch of the bucket's representative roads fastest go into
a table (nasch_set_tuning_table) that the batch planner consults per road.
"""
from __future__ import annotations

import json
import os

from . import build as _build
from . import nasch as NS

CACHE = os.path.join(_build.BUILD, "autotune.json")
K_CANDIDATES = (1, 2, 4, 8, 16, 32)
DENSITIES = (0.02, 0.05, 0.1, 0.15, 0.2, 0.3, 0.45, 0.6, 0.8)


def crossover(densities, agent_rate, grid_rate) -> float:
    """Density where the faster layout changes from agent to grid.

    Rates are vehicle-updates/s at each density.  Returns the midpoint of the
    first adjacent pair where grid overtakes agent for good (the grid stays
    faster at every higher density); 1.0 if agent is always faster, 0.0 if
    grid always is."""
    pts = list(zip(densities, agent_rate, grid_rate))
    pts.sort()
    faster_grid = [g > a for _, a, g in pts]
    if not any(faster_grid):
        return 1.0
    if all(faster_grid):
        return 0.0
    # last density where agent is faster; grid must win from there on
    last_agent = max(i for i, fg in enumerate(faster_grid) if not fg)
    if last_agent + 1 >= len(pts):
        return 1.0
    return 0.5 * (pts[last_agent][0] + pts[last_agent + 1][0])


def _time_road(torch, stream, L, N, layout, k, steps, vmax=5, p=0.13):
    with NS.Road(L, N, vmax, p, 1, 0, layout=layout, k=k, tile=512 if layout == "agent" else 8192,
                 stream=stream) as r:
        r.run(max(k, 2))
        r.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r.run(steps)
        b.record(stream)
        b.synchronize()
        return N * steps / (a.elapsed_time(b) / 1e3)


def tune(L: int = 1 << 24, steps: int = 64, verbose: bool = False) -> dict:
    """Time the candidates on this GPU; returns the chosen settings and the
    measurements (vehicle-updates/s)."""
    import torch
    stream = torch.cuda.Stream()
    res = {"L": L, "steps": steps, "k": {}, "layout": {}}
    best = {}
    for layout, rho in (("agent", 1 / 16), ("grid", 0.5)):
        rates = {}
        for k in K_CANDIDATES:
            n_steps = max(steps, 2 * k) // k * k
            rates[k] = _time_road(torch, stream, L, int(rho * L), layout, k, n_steps)
            if verbose:
                print(f"{layout} k={k}: {rates[k]:.3e}")
        res["k"][layout] = {str(k): v for k, v in rates.items()}
        best[layout] = max(rates, key=rates.get)
    agent_rate, grid_rate = [], []
    for rho in DENSITIES:
        N = max(1, int(rho * L))
        ka, kg = best["agent"], best["grid"]
        agent_rate.append(_time_road(torch, stream, L, N, "agent", ka, max(steps, 2 * ka) // ka * ka))
        grid_rate.append(_time_road(torch, stream, L, N, "grid", kg, max(steps, 2 * kg) // kg * kg))
        if verbose:
            print(f"rho={rho}: agent {agent_rate[-1]:.3e} grid {grid_rate[-1]:.3e}")
    res["layout"] = {"densities": list(DENSITIES), "agent": agent_rate, "grid": grid_rate}
    res["k_agent"] = best["agent"]
    res["k_grid"] = best["grid"]
    res["rho_star"] = crossover(DENSITIES, agent_rate, grid_rate)
    return res


def _key() -> str:
    import torch
    lib = _build.LIB
    stamp = int(os.path.getmtime(lib)) if os.path.exists(lib) else 0
    return f"{torch.cuda.get_device_name(0)}|{stamp}"


def apply(settings: dict) -> None:
    NS.set_tuning(settings["rho_star"], settings["k_agent"], settings["k_grid"])


def load_or_tune(force: bool = False, verbose: bool = False) -> dict:
    """Apply cached settings for this GPU and build, timing them first if needed."""
    key = _key()
    cache = {}
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if force or key not in cache:
        cache[key] = tune(verbose=verbose)
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    apply(cache[key])
    return cache[key]


# --------------------------------------------------------------------------- per-road tuning of batches
# Buckets of roads: decades of L over the uneven ensemble's range, three
# density bands and the ensemble's maximum velocities.  Each bucket gets the
# layout, fusion depth and (grid) tile that ran its representative batch
# fastest; the table goes to nasch_set_tuning_table, which batches and
# servers consult per road.
L_EDGES = (1_000, 10_000, 100_000, 1_000_000, 10_000_001)
RHO_EDGES = (0.0, 0.2, 0.4, 1.0001)
VMAX_SET = (3, 5, 8)
BUCKET_CANDIDATES = ([("agent", k, 0) for k in (4, 8, 16)] +
                     [("grid", k, t) for k in (4, 8, 16) for t in (0, 8192)])
BUCKET_CACHE = os.path.join(_build.BUILD, "autotune_buckets.json")


def buckets():
    """Every (L, density, vmax) bucket: dicts with L_min, L_max, rho_min,
    rho_max, vmax."""
    out = []
    for i in range(len(L_EDGES) - 1):
        for j in range(len(RHO_EDGES) - 1):
            for v in VMAX_SET:
                out.append(dict(L_min=L_EDGES[i], L_max=L_EDGES[i + 1], rho_min=RHO_EDGES[j],
                                rho_max=RHO_EDGES[j + 1], vmax=v))
    return out


def representative_roads(b: dict, cells: int = 1 << 24, p: float = 0.25) -> list[dict]:
    """Roads at the bucket's middle (geometric in L), enough of them to hold
    about `cells` cells (at most 512)."""
    L = int(round((b["L_min"] * min(b["L_max"], 10**7)) ** 0.5))
    rho = 0.5 * (b["rho_min"] + min(b["rho_max"], 1.0))
    N = max(1, min(L, int(round(rho * L))))
    n = max(1, min(512, cells // L))
    return [dict(L=L, N=N, vmax=b["vmax"], p=p, seed=1, road_id=i) for i in range(n)]


def time_batch(roads: list[dict], steps: int, stream=None) -> float:
    """Vehicle-updates/s of one batched job (GPU time after the start states)."""
    with NS.Batch(roads, [steps] * len(roads), stream=stream) as b:
        b.wait()
        sec = b.info().run_seconds
    return sum(r["N"] for r in roads) * steps / sec


def entry(b: dict, layout: str, k: int, tile: int) -> dict:
    return dict(L_min=b["L_min"], L_max=b["L_max"], rho_min=b["rho_min"], rho_max=b["rho_max"],
                vmax_min=b["vmax"], vmax_max=b["vmax"], draw=-1, layout=layout, k=k,
                tile=(tile or 2048) if layout == "grid" else 0)


def tune_buckets(bs=None, steps: int = 64, repeats: int = 2, verbose: bool = False) -> dict:
    """Time every candidate on each bucket's representative batch; returns
    {"entries": table, "timings": per bucket}.  The best of `repeats` runs
    counts for each candidate."""
    import torch
    stream = torch.cuda.Stream()
    table, timings = [], []
    for b in (bs or buckets()):
        roads = representative_roads(b)
        rates = {}
        for layout, k, tile in BUCKET_CANDIDATES:
            rs = [dict(r, layout=layout, k=k, tile=tile) for r in roads]
            rates[(layout, k, tile)] = max(time_batch(rs, steps, stream) for _ in range(repeats))
        best = max(rates, key=rates.get)
        table.append(entry(b, *best))
        timings.append({"bucket": b, "roads": len(roads), "L": roads[0]["L"], "N": roads[0]["N"],
                        "rates": {f"{l}/k{k}/t{t}": v for (l, k, t), v in rates.items()},
                        "best": "/".join(map(str, best))})
        if verbose:
            print(b, best, f"{rates[best]:.3e}")
    return {"entries": table, "timings": timings}


def load_or_tune_buckets(force: bool = False, verbose: bool = False) -> dict:
    """Apply the cached per-bucket table for this GPU and build, timing it
    first if needed."""
    key = _key()
    cache = {}
    if os.path.exists(BUCKET_CACHE):
        try:
            with open(BUCKET_CACHE) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    if force or key not in cache:
        cache[key] = tune_buckets(verbose=verbose)
        os.makedirs(os.path.dirname(BUCKET_CACHE), exist_ok=True)
        with open(BUCKET_CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    NS.set_tuning_table(cache[key]["entries"])
    return cache[key]
