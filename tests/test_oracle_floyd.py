"""Pins for the oracle's initial positions (Handout, "Starter Code": cars
start from random positions on the ring), drawn by Floyd's algorithm
(Bentley & Floyd, CACM 1987) from Philox draws with tag 1.

Floyd's algorithm returns every N-subset of the L cells with probability
1 / C(L, N); the checks are that law (chi^2 over all subsets of small rings),
the structure of the output, and the degenerate sizes.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("L,N", [(1, 1), (1, 0), (10, 10), (1000, 200), (2**20, 2**16), (2**26, 2**22),
                                 (2**31, 5), (17, 16)])
def test_structure(L, N):
    x = O.floyd_init(L, N, seed=1)
    assert len(x) == N
    assert np.all((x >= 0) & (x < L))
    assert np.all(np.diff(x.astype(np.int64)) > 0)   # sorted, distinct
    if N == L:
        assert np.array_equal(x, np.arange(L))


@pytest.mark.parametrize("L,N,road", [(6, 3, 0), (5, 2, 7), (7, 1, 0), (6, 5, 3)])
def test_every_subset_equally_likely(L, N, road):
    subsets = {s: i for i, s in enumerate(itertools.combinations(range(L), N))}
    counts = np.zeros(len(subsets), dtype=np.int64)
    S = 60000
    for seed in range(S):
        counts[subsets[tuple(int(c) for c in O.floyd_init(L, N, seed, road))]] += 1
    exp = S / len(subsets)
    chi2 = float(np.sum((counts - exp) ** 2) / exp)
    dof = len(subsets) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof) + 10, (chi2, dof, counts)


def test_seed_and_road_change_the_sample():
    a = O.floyd_init(10**6, 1000, seed=1, road=0)
    assert not np.array_equal(a, O.floyd_init(10**6, 1000, seed=2, road=0))
    assert not np.array_equal(a, O.floyd_init(10**6, 1000, seed=1, road=1))
    assert np.array_equal(a, O.floyd_init(10**6, 1000, seed=1, road=0))


def test_reference_case_density_spread():
    """The handout's reference case (200 cars on 1000 cells): positions spread
    over the whole ring (Kolmogorov-Smirnov distance to uniform, pooled over
    seeds)."""
    xs = np.concatenate([O.floyd_init(1000, 200, seed=s) for s in range(200)]) / 1000.0
    xs.sort()
    ecdf = np.arange(1, len(xs) + 1) / len(xs)
    ks = float(np.max(np.abs(ecdf - xs)))
    assert ks < 1.63 / math.sqrt(len(xs)) * 2
