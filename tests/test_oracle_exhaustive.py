"""Exhaustive pin of the oracle's step rules on tiny rings.

The model's one step (Handout, "The Nagel-Schreckenberg traffic model",
rules 1-4) is a deterministic function of the state and of the outcomes of
the N independent Bernoulli(p) trials of rule 3.  On every ring of L <= 7
cells, for every number of cars, every placement, every velocity vector
with entries <= vmax and every one of the 2^N trial outcomes, the oracle's
masked step must equal the rules stated here a second way: the gap is found
by scanning the cells ahead for the first occupied one (not by subtracting
positions), and the move is taken on the cell grid.  Then the oracle's keyed
step must be the masked step for the outcomes its Philox draws imply, and
over many seeds the keyed successors of a state must follow the one-step
distribution that the enumeration gives, p^k (1-p)^(N-k) per outcome.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O


def all_states(L, N, vmax):
    """Every (placement, velocities, trial outcomes) of N cars on L cells:
    arrays x, v, slow of shape (count, N), cars in increasing cell order."""
    places = np.array(list(itertools.combinations(range(L), N)), dtype=np.int32)
    vels = np.array(list(itertools.product(range(vmax + 1), repeat=N)), dtype=np.uint8)
    masks = np.array(list(itertools.product((0, 1), repeat=N)), dtype=np.uint8)
    P, V, M = len(places), len(vels), len(masks)
    x = np.repeat(places, V * M, axis=0)
    v = np.tile(np.repeat(vels, M, axis=0), (P, 1))
    slow = np.tile(masks, (P * V, 1))
    return x, v, slow


def rules_by_scanning(L, x, v, slow, vmax):
    """Rules 1-4 on the cell grid: occupancy of every state's cells, the gap
    of each car = empty cells before the first occupied cell ahead (a car
    alone on the ring sees the L - 1 others), then accelerate, brake to the
    gap, slow down by one if the trial succeeded and the car moves, move."""
    S, N = x.shape
    rows = np.arange(S)[:, None]
    occ = np.zeros((S, L), dtype=bool)
    occ[rows, x] = True
    gap = np.full((S, N), L - 1, dtype=np.int64)
    found = np.zeros((S, N), dtype=bool)
    for j in range(1, L):
        hit = occ[rows, (x.astype(np.int64) + j) % L] & ~found
        gap[hit] = j - 1
        found |= hit
    vel = np.minimum(v.astype(np.int64) + 1, vmax)          # rule 1
    vel = np.minimum(vel, gap)                               # rule 2
    vel = np.where((slow != 0) & (vel > 0), vel - 1, vel)   # rule 3
    nx = (x.astype(np.int64) + vel) % L                      # rule 4
    return nx.astype(np.int32), vel.astype(np.uint8)


CASES = [(L, vmax) for L in range(1, 8) for vmax in (0, 1, 2)] + \
        [(L, 3) for L in range(1, 7)] + [(L, 5) for L in range(1, 6)]


@pytest.mark.parametrize("L,vmax", CASES)
def test_masked_step_equals_rules_on_every_state(L, vmax):
    states = 0
    for N in range(1, L + 1):
        x, v, slow = all_states(L, N, vmax)
        ox, ov = O.agent_step_masked(L, x, v, slow, vmax)
        wx, wv = rules_by_scanning(L, x, v, slow, vmax)
        assert np.array_equal(ov, wv), (L, N, vmax, "velocities")
        assert np.array_equal(ox, wx), (L, N, vmax, "positions")
        # no two cars share a cell, and the cyclic order is kept: the new
        # positions, read from the car that was first, are a rotation of an
        # increasing sequence (at most one descent round the ring)
        srt = np.sort(ox, axis=1)
        assert np.all(np.diff(srt, axis=1) > 0), (L, N, vmax, "shared cell")
        descents = (np.diff(np.concatenate([ox, ox[:, :1]], axis=1), axis=1) < 0).sum(axis=1)
        assert np.all(descents <= 1 if N > 1 else descents == 0), (L, N, vmax, "cyclic order")
        states += len(x)
    # every placement x velocities x outcomes was visited: sum_N C(L,N) (2(vmax+1))^N
    assert states == (1 + 2 * (vmax + 1)) ** L - 1


def _keyed_outcomes(x, step, road, seed, p):
    """The rule-3 outcome each car's keyed draw implies: word 0 of Philox of
    counter (cell, step, road, 0) below ceil(p 2^32)."""
    ctr = np.stack([np.asarray(x, np.uint32), np.full(len(x), step, np.uint32),
                    np.full(len(x), road, np.uint32), np.zeros(len(x), np.uint32)], axis=1)
    w0 = O.philox_many(ctr, seed)[:, 0].astype(np.uint64)
    return (w0 < np.uint64(O.slow_threshold(p))).astype(np.uint8)


@pytest.mark.parametrize("L,N,vmax,p", [(7, 3, 2, 0.4), (50, 20, 5, 0.13), (1000, 200, 5, 0.13),
                                        (300, 299, 3, 0.7), (64, 1, 5, 0.5)])
def test_keyed_step_is_masked_step_of_its_draws(L, N, vmax, p):
    rng = np.random.default_rng(L * 1000 + N)
    for trial in range(20):
        seed = int(rng.integers(1, 2**63))
        road = int(rng.integers(0, 2**32))
        step = int(rng.integers(0, 2**32))
        x = np.sort(rng.choice(L, N, replace=False)).astype(np.int32)
        v = rng.integers(0, vmax + 1, N).astype(np.uint8)
        kx, kv, ksv, kcr = O.agent_run(L, x, v, vmax, p, seed, road, step, 1)
        slow = _keyed_outcomes(x, step, road, seed, p)
        mx, mv = O.agent_step_masked(L, x[None], v[None], slow[None], vmax)
        assert np.array_equal(kx, mx[0]) and np.array_equal(kv, mv[0]), trial
        assert int(ksv[0]) == int(mv[0].astype(np.int64).sum())
        assert int(kcr[0]) == int((x.astype(np.int64) + mv[0] >= L).sum())
        gc, _, _ = O.grid_run(O.agent_to_grid(L, x, v), vmax, p, seed, road, step, 1)
        assert np.array_equal(gc, O.agent_to_grid(L, mx[0], mv[0])), trial


@pytest.mark.parametrize("L,x,v,vmax,p", [(6, [0, 2, 3], [1, 0, 2], 2, 0.3),
                                          (7, [0, 1, 4, 5], [2, 1, 0, 2], 2, 0.5),
                                          (5, [1, 3], [5, 1], 5, 0.13)])
def test_keyed_successors_follow_the_enumerated_distribution(L, x, v, vmax, p):
    """Enumerate the 2^N trial outcomes of one state into its successor
    distribution; the oracle's keyed step over 20000 seeds must match it
    (chi-squared, about five standard deviations)."""
    x = np.array(x, np.int32)
    v = np.array(v, np.uint8)
    N = len(x)
    masks = np.array(list(itertools.product((0, 1), repeat=N)), dtype=np.uint8)
    mx, mv = O.agent_step_masked(L, np.tile(x, (len(masks), 1)), np.tile(v, (len(masks), 1)), masks, vmax)
    prob = {}
    for m, a, b in zip(masks, mx, mv):
        k = int(m.sum())
        key = (a.tobytes(), b.tobytes())
        prob[key] = prob.get(key, 0.0) + p ** k * (1 - p) ** (N - k)
    assert math.isclose(sum(prob.values()), 1.0)
    S = 20000
    counts = dict.fromkeys(prob, 0)
    for seed in range(1, S + 1):
        kx, kv, _, _ = O.agent_run(L, x, v, vmax, p, seed, 0, 0, 1)
        key = (kx.tobytes(), kv.tobytes())
        assert key in counts, "a keyed successor that no trial outcome gives"
        counts[key] += 1
    keys = list(prob)
    exp = np.array([prob[k] * S for k in keys])
    obs = np.array([counts[k] for k in keys])
    dof = len(keys) - 1
    assert dof >= 1
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < dof + 5 * math.sqrt(2 * dof) + 10, (chi2, dof, obs, exp)
