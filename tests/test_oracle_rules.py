"""Pins for the oracle's NaSch step (Handout, "The Nagel-Schreckenberg traffic
model", rules 1-4), in both representations ("Concepts Covered": grid and
agent-based), on the ring of "Starter Code".

What pins it, none of which is the oracle re-typed:
  * hand-worked steps (tests/golden/*.txt);
  * vmax = 1, p = 0 is the elementary cellular automaton rule 184;
  * p = 0 from an evenly spaced start below density 1/(vmax+1): closed-form
    positions and flux rho * vmax (the handout: without randomness the
    pattern is preserved);
  * conservation laws and bounds that hold at every step;
  * the grid and agent forms are separate codes and must agree;
  * the one-step distribution over seeds is the product of independent
    Bernoulli(p) slowdowns between the p = 0 and p = 1 successors (chi^2);
  * the exact vmax = 1 flux 0.5 * (1 - sqrt(1 - 4 (1-p) rho (1-rho)))
    (Schreckenberg, Schadschneider, Nagel & Ito, PRE 51, 1995);
  * the assignment's reproducibility requirement: the OpenMP build equals
    the serial build at any thread count.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import _golden


def _floyd_state(L, N, seed, road=0):
    x = O.floyd_init(L, N, seed, road)
    return x, np.zeros(N, dtype=np.uint8)


@pytest.mark.parametrize("name", _golden.ALL)
def test_hand_worked_fixtures_agent(name):
    fx = _golden.load(name)
    x, v = fx["x"], fx["v"]
    prev = 0
    for t in _golden.steps(fx):
        x, v, sv, cr = O.agent_run(fx["L"], x, v, fx["vmax"], fx["p"], seed=99, step0=prev, T=t - prev)
        assert x.tolist() == fx[f"x@{t}"], (name, t)
        assert v.tolist() == fx[f"v@{t}"], (name, t)
        assert int(sv[-1]) == fx[f"sum_v@{t}"]
        assert int(cr[-1]) == fx[f"crossings@{t}"]
        prev = t


@pytest.mark.parametrize("name", _golden.ALL)
def test_hand_worked_fixtures_grid(name):
    fx = _golden.load(name)
    L = fx["L"]
    cells = O.agent_to_grid(L, fx["x"], fx["v"])
    prev = 0
    for t in _golden.steps(fx):
        cells, sv, cr = O.grid_run(cells, fx["vmax"], fx["p"], seed=99, step0=prev, T=t - prev)
        want = O.agent_to_grid(L, fx[f"x@{t}"], fx[f"v@{t}"])
        assert np.array_equal(cells, want), (name, t)
        assert int(sv[-1]) == fx[f"sum_v@{t}"]
        assert int(cr[-1]) == fx[f"crossings@{t}"]
        prev = t


def _rule184(occ):
    """Wolfram code 184 on a periodic row: new = bit (4*left + 2*centre + right) of 184."""
    left, right = np.roll(occ, 1), np.roll(occ, -1)
    idx = 4 * left + 2 * occ + right
    return (184 >> idx) & 1


@pytest.mark.parametrize("seed", range(6))
def test_vmax1_p0_is_rule_184(seed):
    rng = np.random.default_rng(seed)
    L = 97
    occ = (rng.random(L) < rng.uniform(0.1, 0.9)).astype(np.int64)
    occ[0] = 1
    x = np.flatnonzero(occ).astype(np.int32)
    v = rng.integers(0, 2, len(x)).astype(np.uint8)
    cells = O.agent_to_grid(L, x, v)
    for step in range(40):
        x, v, _, _ = O.agent_run(L, x, v, 1, 0.0, seed=1, step0=step, T=1)
        cells, _, _ = O.grid_run(cells, 1, 0.0, seed=1, step0=step, T=1)
        occ = _rule184(occ)
        agent_occ = np.zeros(L, dtype=np.int64)
        agent_occ[x] = 1
        assert np.array_equal(agent_occ, occ)
        assert np.array_equal((cells >= 0).astype(np.int64), occ)


@pytest.mark.parametrize("vmax,spacing,n", [(5, 6, 50), (5, 9, 40), (2, 3, 33), (8, 12, 10), (1, 2, 64)])
def test_p0_even_start_closed_form(vmax, spacing, n):
    """Evenly spaced cars at density 1/spacing <= 1/(vmax+1), all v=0, p=0: every
    car accelerates by one per step up to vmax and never brakes, so after t
    steps each car has moved D(t) = sum_{s=1..t} min(s, vmax) and the flux is
    rho * vmax once t >= vmax."""
    L = spacing * n
    x0 = np.arange(n, dtype=np.int64) * spacing
    x, v, sv, cr = O.agent_run(L, x0, np.zeros(n), vmax, 0.0, seed=5, T=3 * vmax + 7)
    T = 3 * vmax + 7
    D = sum(min(s, vmax) for s in range(1, T + 1))
    assert np.array_equal(x, (x0 + D) % L)
    assert np.all(v == vmax)
    assert [int(s) for s in sv] == [n * min(t + 1, vmax) for t in range(T)]
    # flux J = sum_v / L = rho * vmax after vmax steps
    assert all(int(s) * spacing == L * vmax for s in sv[vmax - 1:])
    cells = O.agent_to_grid(L, x0.astype(np.int32), np.zeros(n, np.uint8))
    cells, sv2, cr2 = O.grid_run(cells, vmax, 0.0, seed=5, T=T)
    assert np.array_equal(cells, O.agent_to_grid(L, x, v))
    assert np.array_equal(sv, sv2) and np.array_equal(cr, cr2)


def _check_invariants(L, vmax, x0, x1, v1, sv, cr):
    N = len(x0)
    assert len(x1) == N
    assert np.all((x1 >= 0) & (x1 < L))
    assert len(np.unique(x1)) == N, "two cars on one cell"
    assert np.all(v1 <= vmax)
    disp = (x1.astype(np.int64) - x0.astype(np.int64)) % L
    assert np.array_equal(disp, v1.astype(np.int64)), "moved by v"
    assert int(sv) == int(v1.astype(np.int64).sum())
    assert int(cr) == int(np.sum(x0.astype(np.int64) + v1 >= L))
    if N >= 2:
        # cyclic order kept: exactly one descent going round the ring
        nxt = np.roll(x1, -1)
        assert int(np.sum(nxt < x1)) == 1


CASES = [  # (L, N, vmax, p)
    (1000, 200, 5, 0.13),          # the handout's reference case (Fig. 1 caption)
    (500, 300, 2, 0.2),            # the handout's example parameter file values
    (64, 1, 5, 0.3), (9, 9, 3, 0.5), (10, 9, 2, 0.4), (37, 5, 20, 0.9),
    (257, 128, 8, 0.0), (257, 128, 8, 1.0), (3, 2, 127, 0.5), (1, 1, 3, 0.5),
    (100, 30, 0, 0.5),
]


@pytest.mark.parametrize("L,N,vmax,p", CASES)
def test_invariants_and_grid_equals_agent(L, N, vmax, p):
    x, v = _floyd_state(L, N, seed=3, road=2)
    cells = O.agent_to_grid(L, x, v)
    for step in range(60):
        x1, v1, sv, cr = O.agent_run(L, x, v, vmax, p, seed=3, road=2, step0=step, T=1)
        _check_invariants(L, vmax, x, x1, v1, sv[0], cr[0])
        cells, gsv, gcr = O.grid_run(cells, vmax, p, seed=3, road=2, step0=step, T=1)
        assert np.array_equal(cells, O.agent_to_grid(L, x1, v1))
        assert gsv[0] == sv[0] and gcr[0] == cr[0]
        x, v = x1, v1


def test_multi_step_equals_repeated_single_steps_and_resume():
    L, N, vmax, p = 700, 150, 5, 0.25
    x, v = _floyd_state(L, N, seed=11)
    xa, va, sa, ca = O.agent_run(L, x, v, vmax, p, seed=11, T=200)
    xb, vb = x, v
    sb, cb = [], []
    bounds = [0, 37, 38, 120, 200]
    for a, b in zip(bounds[:-1], bounds[1:]):
        xb, vb, s, c = O.agent_run(L, xb, vb, vmax, p, seed=11, step0=a, T=b - a)
        sb += list(s)
        cb += list(c)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    assert list(sa) == sb and list(ca) == cb


def test_draws_depend_on_seed_road_and_step():
    L, N, vmax, p = 1000, 200, 5, 0.5
    x, v = _floyd_state(L, N, seed=1)
    base = O.agent_run(L, x, v, vmax, p, seed=1, road=0, step0=0, T=20)[0]
    for kw in (dict(seed=2), dict(road=1), dict(step0=1)):
        args = dict(seed=1, road=0, step0=0)
        args.update(kw)
        other = O.agent_run(L, x, v, vmax, p, T=20, **args)[0]
        assert not np.array_equal(base, other), kw


def _one_step_outcomes(L, x, v, vmax):
    """Successors with no slowdown (p=0) and with every possible slowdown (p=1)."""
    x0, v0, _, _ = O.agent_run(L, x, v, vmax, 0.0, seed=0, T=1)
    x1, v1, _, _ = O.agent_run(L, x, v, vmax, 1.0, seed=0, T=1)
    return v0, v1


@pytest.mark.parametrize("L,x,v,vmax", [
    (8, [0, 2, 5], [1, 2, 0], 3),
    (7, [1, 2, 4, 6], [0, 1, 1, 0], 2),
    (6, [0, 3], [2, 2], 5),
    (5, [0, 1, 2, 3, 4], [1, 1, 1, 1, 1], 2),
])
def test_one_step_distribution_matches_enumeration(L, x, v, vmax):
    """Over many seeds each car independently takes its p=1 velocity with
    probability p (when that differs from its p=0 velocity): compare the
    empirical mask frequencies with p^k (1-p)^(n-k) by chi^2."""
    p = 0.3
    v0, v1 = _one_step_outcomes(L, x, v, vmax)
    free = np.flatnonzero(v0 != v1)
    n = len(free)
    counts = np.zeros(2 ** n, dtype=np.int64)
    S = 20000
    for seed in range(S):
        xs, vs, _, _ = O.agent_run(L, x, v, vmax, p, seed=seed, T=1)
        assert np.all((vs == v0) | (vs == v1))
        assert np.array_equal(xs, (np.asarray(x) + vs) % L)
        mask = 0
        for b, i in enumerate(free):
            if vs[i] == v1[i]:
                mask |= 1 << b
        counts[mask] += 1
    exp = np.array([p ** bin(m).count("1") * (1 - p) ** (n - bin(m).count("1")) for m in range(2 ** n)]) * S
    chi2 = float(np.sum((counts - exp) ** 2 / exp))
    dof = 2 ** n - 1
    if dof == 0:
        assert counts[0] == S
        return
    # 5-sigma-ish bound on chi^2 with dof degrees of freedom
    assert chi2 < dof + 5 * math.sqrt(2 * dof) + 10, (chi2, dof, counts, exp)


@pytest.mark.parametrize("rho,p", [(0.3, 0.5), (0.5, 0.25), (0.1, 0.75)])
def test_vmax1_flux_matches_exact_result(rho, p):
    """vmax = 1 NaSch has the exact stationary flux
    J = (1 - sqrt(1 - 4 (1-p) rho (1-rho))) / 2."""
    L = 20000
    N = int(rho * L)
    x, v = _floyd_state(L, N, seed=21)
    x, v, _, _ = O.agent_run(L, x, v, 1, p, seed=21, T=2000)
    _, _, sv, _ = O.agent_run(L, x, v, 1, p, seed=21, step0=2000, T=3000)
    J = float(sv.astype(np.float64).sum()) / (L * 3000)
    exact = 0.5 * (1 - math.sqrt(1 - 4 * (1 - p) * rho * (1 - rho)))
    assert abs(J - exact) < 0.01 * exact + 2e-4, (J, exact)


@pytest.mark.parametrize("threads", [1, 2, 3, 4, 8])
def test_openmp_build_equals_serial(threads):
    L, N, vmax, p = 5000, 1500, 5, 0.13
    x, v = _floyd_state(L, N, seed=8)
    want = O.agent_run(L, x, v, vmax, p, seed=8, T=100)
    O.set_threads(threads)
    got = O.agent_run(L, x, v, vmax, p, seed=8, T=100, openmp=True)
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
    cells = O.agent_to_grid(L, x, v)
    gw = O.grid_run(cells, vmax, p, seed=8, T=100)
    gg = O.grid_run(cells, vmax, p, seed=8, T=100, openmp=True)
    for a, b in zip(gw, gg):
        assert np.array_equal(a, b)


def test_segments_equal_ring_runs():
    L, N, vmax, p, T = 3000, 700, 5, 0.13, 25
    x, v = _floyd_state(L, N, seed=4, road=9)
    xr, vr, _, _ = O.agent_run(L, x, v, vmax, p, seed=4, road=9, step0=100, T=T)
    for start in (0, 350, N - 50):   # the last window wraps round the ring
        idx = (start + np.arange(120)) % N
        xs, vs = O.agent_segment(L, x[idx], v[idx], vmax, p, seed=4, road=9, step0=100, T=T)
        assert np.array_equal(xs, xr[idx[: 120 - T]])
        assert np.array_equal(vs, vr[idx[: 120 - T]])
    cells = O.agent_to_grid(L, x, v)
    cr, _, _ = O.grid_run(cells, vmax, p, seed=4, road=9, step0=100, T=T)
    for first in (0, 1234, L - 300):
        idx = (first + np.arange(600)) % L
        mid = O.grid_segment(L, cells[idx], first, vmax, p, seed=4, road=9, step0=100, T=T)
        m = T * vmax
        assert np.array_equal(mid, cr[idx[m: 600 - m]])


def test_empty_road_and_zero_steps():
    x, v, sv, cr = O.agent_run(10, [], [], 5, 0.5, seed=1, T=4)
    assert len(x) == 0 and list(sv) == [0] * 4 and list(cr) == [0] * 4
    cells, sv, cr = O.grid_run(np.full(10, -1, np.int8), 5, 0.5, seed=1, T=3)
    assert np.all(cells == -1) and list(sv) == [0] * 3
    x0, v0 = _floyd_state(50, 10, 1)
    x, v, sv, cr = O.agent_run(50, x0, v0, 5, 0.5, seed=1, T=0)
    assert np.array_equal(x, x0) and len(sv) == 0
