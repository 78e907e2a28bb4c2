"""Synthetic workloads shaped like the paper's roads (no method arithmetic).

* ``REFERENCE_CASE``: the handout's reference test case, 200 cars on a
  1000-cell ring, p = 0.13, vmax = 5 (Fig. 1 caption), run for 1000 steps
  from a seeded random start.
* ``LARGE_ROAD``: one ring of 2^31 cells holding 2^27 cars (density 1/16),
  vmax = 5, p = 0.13, 10^4 steps: the "longer and more demanding run" of the
  handout's large test file, whose parameters the paper does not print,
  scaled to a GPU's memory.
* ``EXAMPLE_PARAMS``: the example values of the handout's parameter file
  description (L = 500, T = 500, N = 300, p = 0.2, vmax = 2, seed = 13).
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class RoadSpec:
    name: str
    L: int
    N: int
    vmax: int
    p: float
    T: int
    seed: int = 1
    road_id: int = 0


REFERENCE_CASE = RoadSpec("reference-case L=1000 N=200 vmax=5 p=0.13 T=1000", 1000, 200, 5, 0.13, 1000)
LARGE_ROAD = RoadSpec("large-road L=2^31 N=2^27 vmax=5 p=0.13 T=10^4", 2**31, 2**27, 5, 0.13, 10_000)
EXAMPLE_PARAMS = RoadSpec("example-params L=500 N=300 vmax=2 p=0.2 T=500", 500, 300, 2, 0.2, 500, seed=13)

# Launch configuration the benchmark times on LARGE_ROAD (fusion depth per
# layout); the full-size parity tests run the same.
LARGE_ROAD_K = {"agent": 16, "grid": 8}


# --------------------------------------------------------------------------- batched workloads
import csv as _csv  # noqa: E402
import os as _os  # noqa: E402

_DATA = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "data")

FD_DENSITIES = 64            # densities 0.02 .. 0.90, evenly spaced
FD_PS = (0.0, 0.13, 0.25, 0.5)
FD_L = 10**6
FD_T = 12_000
FD_WARMUP = 2_000


def fd_cars(i: int, L: int = FD_L) -> int:
    """Cars at density index i of the sweep: rho_i = 0.02 + 0.88 i / 63 =
    (1260 + 880 i) / 63000, rounded half up in exact integers, in [1, L]."""
    return max(1, min(L, (L * (1260 + 880 * i) + 31500) // 63000))


def fundamental_diagram_roads(replicas: int = 128, L: int = FD_L, densities: int = FD_DENSITIES, ps=FD_PS,
                              vmax: int = 5):
    """The density sweep: densities x ps x replicas roads of L cells (vmax 5
    by default).  Replica r uses seed r + 1; the road id is the flat index
    (density-major)."""
    roads = []
    for i in range(densities):
        for j, p in enumerate(ps):
            for r in range(replicas):
                roads.append(dict(L=L, N=fd_cars(i, L), vmax=vmax, p=p, seed=r + 1,
                                  road_id=(i * len(ps) + j) * replicas + r))
    return roads


def flux_vmax1(rho: float, p: float) -> float:
    """Steady-state flux of the vmax = 1 model with parallel update
    (Schreckenberg, Schadschneider, Nagel & Ito, Phys. Rev. E 51, 1995):
    J = (1 - sqrt(1 - 4 (1 - p) rho (1 - rho))) / 2."""
    return 0.5 * (1.0 - (1.0 - 4.0 * (1.0 - p) * rho * (1.0 - rho)) ** 0.5)


def _load_table(name: str):
    rows = []
    with open(_os.path.join(_DATA, name)) as f:
        for rec in _csv.DictReader(f):
            thr = int(rec["threshold"])
            row = dict(L=int(rec["L"]), N=int(rec["N"]), vmax=int(rec["vmax"]),
                       p=thr / 2.0**32,   # exact: ceil(p * 2^32) gives back the threshold
                       seed=7 if name.startswith("ensemble") else 11, road_id=int(rec["road_id"]),
                       T=int(rec["T"]))
            if "arrival_micro" in rec:
                row["arrival"] = int(rec["arrival_micro"]) * 1e-6
            rows.append(row)
    return rows


def uneven_ensemble():
    """4096 roads of the seed-7 table: L log-uniform [1e3, 1e7], density
    U[0.05, 0.6], vmax in {3, 5, 8}, p U[0, 0.5), T log-uniform [1e3, 1e5]."""
    return _load_table("ensemble_seed7.csv")


def request_stream():
    """20000 requests of the seed-11 table (same distributions) with unit-rate
    Poisson arrival times (`arrival`, seconds at rate 1)."""
    return _load_table("requests_seed11.csv")


def road_params(row: dict) -> dict:
    """The nasch_params keys of a table row (drops T and arrival)."""
    return {k: row[k] for k in ("L", "N", "vmax", "p", "seed", "road_id")}
