"""Write the integer parameter tables of the uneven ensemble and the request
stream (seeded, synthetic; no method arithmetic).

Each road: L log-uniform on [10^3, 10^7], density rho uniform on [0.05, 0.6],
N = round(rho * L) clamped to [1, L], vmax uniform on {3, 5, 8}, p uniform on
[0, 0.5) stored as its integer slowdown threshold ceil(p * 2^32), T
log-uniform on [10^3, 10^5].  The request stream adds Poisson arrival times
of unit rate (exponential gaps of mean 1, stored in micro-units), to be
scaled by the offered rate.  Floats (log, exp) are used only here, once; the
tables are committed as integers so every machine reads identical roads.

    python -m paper_2309_14311_gb300.data.make_tables
"""
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ENSEMBLE = os.path.join(HERE, "ensemble_seed7.csv")
REQUESTS = os.path.join(HERE, "requests_seed11.csv")
HEADER = "road_id,L,N,vmax,threshold,T"


def draw_roads(rng: np.random.Generator, n: int):
    rows = []
    for i in range(n):
        u = rng.random(5)
        L = int(min(10**7, max(10**3, math.floor(10 ** (3 + 4 * u[0])))))
        rho = 0.05 + 0.55 * u[1]
        N = int(min(L, max(1, round(rho * L))))
        vmax = (3, 5, 8)[min(2, int(3 * u[2]))]
        p = 0.5 * u[3]
        thr = int(math.ceil(p * 2**32))
        T = int(min(10**5, max(10**3, math.floor(10 ** (3 + 2 * u[4])))))
        rows.append((i, L, N, vmax, thr, T))
    return rows


def main():
    rng = np.random.Generator(np.random.PCG64(7))
    with open(ENSEMBLE, "w") as f:
        f.write(HEADER + "\n")
        for r in draw_roads(rng, 4096):
            f.write(",".join(map(str, r)) + "\n")
    rng = np.random.Generator(np.random.PCG64(11))
    roads = draw_roads(rng, 20000)
    gaps = rng.exponential(1.0, len(roads))
    t = np.cumsum(gaps)
    with open(REQUESTS, "w") as f:
        f.write(HEADER + ",arrival_micro\n")
        for r, a in zip(roads, t):
            f.write(",".join(map(str, r)) + f",{int(round(a * 1e6))}\n")


if __name__ == "__main__":
    main()
