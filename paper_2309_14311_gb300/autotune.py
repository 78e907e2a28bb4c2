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
