"""The committed parameter tables of the uneven ensemble (seed 7, 4096 roads)
and the request stream (seed 11, 20000 requests) follow the recipe their
generator states, and the generator reproduces them: L and T log-uniform on
[10^3, 10^7] and [10^3, 10^5], density uniform on [0.05, 0.6] with N =
round(rho L), vmax uniform on {3, 5, 8}, p uniform on [0, 0.5) stored as its
slowdown threshold, and unit-rate Poisson arrivals."""
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
