"""The committed parameter tables of the uneven ensemble (seed 7, 4096 roads)
and the request stream (seed 11, 20000 requests) follow the recipe their
generator states, and the generator reproduces them: L and T log-uniform on
[10^3, 10^7] and [10^3, 10^5], density uniform on [0.05, 0.6] with N =
round(rho L), vmax uniform on {3, 5, 8}, p uniform on [0, 0.5) stored as its
slowdown threshold, and unit-rate Poisson arrivals.  The density sweep's
roads follow its exact integer rounding."""
import math

import numpy as np
import pytest

from paper_2309_14311_gb300.data import make_tables as MT


def load(path):
    return np.loadtxt(path, delimiter=",", skiprows=1, dtype=np.int64)


@pytest.fixture(scope="module")
def tables():
    return load(MT.ENSEMBLE), load(MT.REQUESTS)


def ks_uniform(u):
    """Kolmogorov-Smirnov distance of a sample in [0, 1] from U(0, 1)."""
    u = np.sort(u)
    n = len(u)
    return max(np.max(np.arange(1, n + 1) / n - u), np.max(u - np.arange(n) / n))


@pytest.mark.parametrize("which", [0, 1])
def test_tables_follow_the_recipe(tables, which):
    t = tables[which]
    n = len(t)
    assert n == (4096, 20000)[which]
    road_id, L, N, vmax, thr, T = (t[:, i] for i in range(6))
    assert np.array_equal(road_id, np.arange(n))
    assert L.min() >= 10**3 and L.max() <= 10**7
    assert T.min() >= 10**3 and T.max() <= 10**5
    assert np.all((N >= 1) & (N <= L))
    assert set(np.unique(vmax)) == {3, 5, 8}
    assert np.all((thr >= 0) & (thr < 2**31))            # p < 0.5
    crit = 1.63 / math.sqrt(n)                            # KS critical value at the 1 % level
    assert ks_uniform((np.log10(L) - 3) / 4) < crit + 1e-3   # floor() shifts L down by < 1 cell
    assert ks_uniform((np.log10(T) - 3) / 2) < crit + 1e-3
    assert ks_uniform(thr / 2**31) < crit
    rho = N / L
    big = L >= 10**4                                      # rounding moves rho by < 1e-4 there
    assert ks_uniform((rho[big] - 0.05) / 0.55) < 1.63 / math.sqrt(big.sum()) + 1e-3
    counts = np.array([(vmax == v).sum() for v in (3, 5, 8)])
    assert np.all(np.abs(counts - n / 3) < 4 * math.sqrt(n * 2 / 9))


def test_arrivals_are_unit_rate_poisson(tables):
    a = tables[1][:, 6].astype(np.float64) / 1e6
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert np.all(gaps >= 0)
    n = len(gaps)
    assert abs(gaps.mean() - 1.0) < 4 / math.sqrt(n)
    assert ks_uniform(1.0 - np.exp(-gaps)) < 1.63 / math.sqrt(n)


def test_generator_reproduces_the_tables(tables):
    ens, req = tables
    rng = np.random.Generator(np.random.PCG64(7))
    assert np.array_equal(np.array(MT.draw_roads(rng, 4096), dtype=np.int64), ens)
    rng = np.random.Generator(np.random.PCG64(11))
    roads = np.array(MT.draw_roads(rng, 20000), dtype=np.int64)
    arrival = np.rint(np.cumsum(rng.exponential(1.0, len(roads))) * 1e6).astype(np.int64)
    assert np.array_equal(roads, req[:, :6])
    assert np.array_equal(arrival, req[:, 6])


def test_density_sweep_roads():
    """The density sweep: rho_i = 0.02 + 0.88 i / 63 for i = 0..63, N_i =
    L rho_i rounded half up (computed here with exact rationals), p in
    {0, 0.13, 0.25, 0.5}, 128 replicas with seeds 1..128, road ids the flat
    index, density-major."""
    from fractions import Fraction

    from paper_2309_14311_gb300 import workloads as WL

    roads = WL.fundamental_diagram_roads()
    assert len(roads) == 64 * 4 * 128
    assert [r["road_id"] for r in roads] == list(range(len(roads)))
    for i in range(64):
        rho = Fraction(2, 100) + Fraction(88, 100) * i / 63
        want = math.floor(10**6 * rho + Fraction(1, 2))
        block = roads[i * 512:(i + 1) * 512]
        assert {r["N"] for r in block} == {want}, i
        assert [r["p"] for r in block] == [p for p in (0.0, 0.13, 0.25, 0.5) for _ in range(128)]
        assert [r["seed"] for r in block] == list(range(1, 129)) * 4
        assert all(r["L"] == 10**6 and r["vmax"] == 5 for r in block)
    assert roads[0]["N"] == 20000 and roads[-1]["N"] == 900000
    # a short road rounds half up and stays in [1, L]
    assert WL.fd_cars(0, 25) == 1 and WL.fd_cars(63, 10) == 9 and WL.fd_cars(0, 1) == 1
