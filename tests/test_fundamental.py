"""CPU tests of the fundamental-diagram products (``fundamental.py``): exact
time averages divided once, the replica interval, the closed forms, and a
small sweep run by the oracle."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import fundamental as FD


def test_mean_sd_and_interval_of_known_replicas():
    # four replicas of L = 100 cells over 10 steps: fluxes 1.0, 1.1, 1.2, 0.9
    rs = [FD.ReplicaSum(L=100, N=40, p=0.25, vmax=5, total_sum_v=s, steps=10) for s in (1000, 1100, 1200, 900)]
    (row,) = FD.fd_table(rs)
    assert row["J"] == pytest.approx(1.05, abs=1e-15)
    assert row["v"] == pytest.approx(4200 / (4 * 40 * 10), abs=1e-15)
    sd = math.sqrt(0.05 / 3)                     # squared deviations 0.0025, 0.0025, 0.0225, 0.0225
    assert row["J_sd"] == pytest.approx(sd, rel=1e-12)
    # Student's t, 3 degrees of freedom, two-sided 95 %: 3.182446...
    assert row["J_ci95"] == pytest.approx(3.182446305284263 * sd / 2, rel=1e-6)
    assert "J_theory" not in row and row["replicas"] == 4


def test_sums_are_divided_once_and_exactly():
    # a sum whose float conversion before dividing would round
    big = (1 << 60) + 3
    (row,) = FD.fd_table([FD.ReplicaSum(L=3, N=1, p=0.1, vmax=5, total_sum_v=big, steps=7)])
    assert row["J"] == float(Fraction(big, 21))
    assert row["v"] == float(Fraction(big, 7))


def test_closed_forms():
    # p = 0: min(vmax rho, 1 - rho), exact
    assert FD.theory_flux(Fraction(1, 10), 0.0, 5) == Fraction(1, 2)
    assert FD.theory_flux(Fraction(3, 10), 0.0, 5) == Fraction(7, 10)
    assert FD.theory_flux(Fraction(1, 6), 0.0, 5) == Fraction(5, 6)   # the critical density: both branches
    # vmax = 1: at rho = 1/2, p = 1/2 the root is sqrt(1/2)
    assert FD.theory_flux(0.5, 0.5, 1) == pytest.approx((1 - math.sqrt(0.5)) / 2, rel=1e-15)
    # vmax = 1, p = 0 falls on the first form: min(rho, 1 - rho)
    assert FD.theory_flux(Fraction(1, 4), 0.0, 1) == Fraction(1, 4)
    assert FD.theory_flux(Fraction(1, 4), 0.3, 5) is None


def test_rows_sorted_by_p_then_density_and_grouped():
    rs = [FD.ReplicaSum(100, n, p, 5, 10 * n, 10) for p in (0.5, 0.0) for n in (30, 10) for _ in range(2)]
    rows = FD.fd_table(rs)
    assert [(r["p"], r["N"]) for r in rows] == [(0.0, 10), (0.0, 30), (0.5, 10), (0.5, 30)]
    assert all(r["replicas"] == 2 for r in rows)
    with pytest.raises(ValueError):
        FD.fd_table([FD.ReplicaSum(100, 10, 0.1, 5, 5, 10), FD.ReplicaSum(100, 10, 0.1, 5, 5, 11)])


def _oracle_sweep(L, densities, ps, vmax, replicas, T, warm):
    out = []
    for rho in densities:
        N = int(round(rho * L))
        for p in ps:
            for r in range(replicas):
                x0 = O.floyd_init(L, N, r + 1, 0)
                _, _, sv, _ = O.agent_run(L, x0, np.zeros(N, np.uint8), vmax, p, r + 1, 0, 0, T)
                out.append(FD.ReplicaSum(L, N, p, vmax, int(sv[warm:].sum()), T - warm))
    return out


def test_small_oracle_sweep_against_closed_forms():
    """A 2000-cell sweep run by the oracle: for p = 0 away from the critical
    density 1/(vmax+1) the deterministic steady state is reached and the
    flux equals min(vmax rho, 1 - rho) exactly; for vmax = 1 the flux lies
    near the exact stationary value."""
    rows = FD.fd_table(_oracle_sweep(2000, (0.05, 0.1, 0.3, 0.6), (0.0,), 5, 3, 3000, 1000))
    for r in rows:
        assert r["J_minus_theory"] == 0.0, r
    rows = FD.fd_table(_oracle_sweep(2000, (0.1, 0.3, 0.5, 0.8), (0.25, 0.5), 1, 4, 3000, 1000))
    for r in rows:
        assert abs(r["J_minus_theory"]) < 0.01 * r["J_theory"] + 3 * r["J_ci95"], r
    s = FD.summary(rows)
    assert s["theory_points"] == len(rows) == 8
