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
LARGE_ROAD_K = {"agent": 4, "grid": 8}
