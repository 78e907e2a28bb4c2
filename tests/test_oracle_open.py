"""Pins of the oracle's open road (the handout's "Variations": other boundary
conditions; entry before cell 0 with probability alpha, exit after cell L-1
open with probability beta).  Hand-worked steps, and what the reading fixes
whatever the draws: cars that only leave, a road that only fills, the car
count changing by the exits and at most one entry per step, free
acceleration of a car alone, and the interior of the road stepping exactly
as on the ring."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import _golden

FIXTURES = ["open_entry_exit_L10.txt", "open_closed_exit_L6.txt", "open_p1_L5.txt"]


def cells_of(L, x, v):
    c = np.full(L, -1, np.int8)
    c[np.asarray(x, dtype=np.int64)] = np.asarray(v, dtype=np.int8)
    return c


@pytest.mark.parametrize("name", FIXTURES)
def test_hand_worked_steps(name):
    fx = _golden.load(name)
    L = fx["L"]
    c = cells_of(L, fx["x"], fx["v"])
    for t in _golden.steps(fx):
        c, sv, cr = O.open_run(c, fx["vmax"], fx["p"], fx["alpha"], fx["beta"], seed=3, road=0, step0=t - 1, T=1)
        assert np.array_equal(c, cells_of(L, fx[f"x@{t}"], fx[f"v@{t}"])), (name, t)
        assert int(sv[0]) == fx[f"sum@{t - 1}"] and int(cr[0]) == fx[f"left@{t - 1}"], (name, t)


def test_cars_only_leave_when_nothing_enters():
    L, N = 300, 120
    c = O.agent_to_grid(L, O.floyd_init(L, N, 5, 0), np.zeros(N, np.uint8))
    c, sv, cr = O.open_run(c, 5, 0.3, 0.0, 1.0, seed=5, road=0, step0=0, T=3 * L)
    assert not (c >= 0).any()
    assert int(cr.sum()) == N


def test_road_fills_when_nothing_leaves():
    L = 40
    c = np.full(L, -1, np.int8)
    c, sv, cr = O.open_run(c, 3, 0.4, 1.0, 0.0, seed=2, road=1, step0=0, T=20 * L)
    assert (c >= 0).all() and not cr.any()


@pytest.mark.parametrize("alpha,beta,p", [(0.3, 0.7, 0.13), (0.9, 0.2, 0.5), (0.5, 0.5, 0.0)])
def test_car_count_changes_by_exits_and_one_entry(alpha, beta, p):
    L = 500
    c = O.agent_to_grid(L, O.floyd_init(L, 100, 9, 2), np.zeros(100, np.uint8))
    n = int((c >= 0).sum())
    for t in range(200):
        c, sv, cr = O.open_run(c, 5, p, alpha, beta, seed=9, road=2, step0=t, T=1)
        n2 = int((c >= 0).sum())
        entered = n2 - n + int(cr[0])
        assert entered in (0, 1)
        assert (c[c >= 0] <= 5).all()
        n = n2


def test_free_acceleration_of_a_car_alone():
    # p = 0, exit open: x_{t+1} = x_t + min(v_t + 1, vmax) until it leaves
    L, vmax, x, v = 60, 4, 3, 0
    c = cells_of(L, [x], [v])
    t = 0
    while True:
        c, sv, cr = O.open_run(c, vmax, 0.0, 0.0, 1.0, seed=1, road=0, step0=t, T=1)
        v = min(v + 1, vmax)
        x += v
        assert int(sv[0]) == v
        if x >= L:
            assert int(cr[0]) == 1 and not (c >= 0).any()
            break
        assert np.array_equal(c, cells_of(L, [x], [v]))
        t += 1


def test_interior_steps_as_on_the_ring():
    # cars far from both ends see the same leaders and draws as on a ring
    L, vmax = 400, 5
    rng = np.random.default_rng(4)
    x = np.sort(rng.choice(np.arange(50, 350), 60, replace=False))
    v = rng.integers(0, vmax + 1, 60).astype(np.uint8)
    c = cells_of(L, x, v)
    ring, _, _ = O.grid_run(c, vmax, 0.25, 7, 3, 11, 1)
    opened, _, _ = O.open_run(c, vmax, 0.25, 0.0, 1.0, seed=7, road=3, step0=11, T=1)
    assert np.array_equal(ring[40:300], opened[40:300])
