"""Fundamental-diagram products of a density sweep: the time-averaged flux and
mean velocity per (density, p), their spread over replicas, and the closed
forms they can be checked against.

The flux of one road over the averaging window of `steps` steps is
J = (sum over the window of sum_v) / (L * steps), the mean velocity
v = (the same sum) / (N * steps): the per-step integers the library reports
(sum_v, the velocities used by the moves) summed exactly and divided once.
Closed forms:
  * p = 0 (deterministic model), steady state from any start:
    J = min(vmax * rho, 1 - rho);
  * vmax = 1, any p (Schreckenberg, Schadschneider, Nagel & Ito, Phys. Rev.
    E 51, 1995): J = (1 - sqrt(1 - 4 (1 - p) rho (1 - rho))) / 2.
Plain host arithmetic on the library's outputs; nothing here steps a road.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from fractions import Fraction


@dataclass(frozen=True)
class ReplicaSum:
    """One road of the sweep: its size, p, and the exact sum of sum_v over
    its averaging window of `steps` steps."""
    L: int
    N: int
    p: float
    vmax: int
    total_sum_v: int
    steps: int


def t_quantile_975(dof: int) -> float:
    """Two-sided 95 % quantile of Student's t with `dof` degrees of freedom
    (the normal 1.96 for large dof)."""
    if dof < 1:
        return float("nan")
    try:
        from scipy.stats import t
        return float(t.ppf(0.975, dof))
    except Exception:   # no scipy: the normal quantile, good for dof >= 30
        return 1.959963984540054


def theory_flux(rho: Fraction | float, p: float, vmax: int):
    """The closed-form steady-state flux where one is known, else None.
    p = 0 returns an exact Fraction when rho is one."""
    if p == 0.0:
        return min(vmax * rho, 1 - rho)
    if vmax == 1:
        r = float(rho)
        return 0.5 * (1.0 - math.sqrt(1.0 - 4.0 * (1.0 - p) * r * (1.0 - r)))
    return None


def fd_table(replicas: list[ReplicaSum]) -> list[dict]:
    """Group replicas by (L, N, p, vmax) and report per group, sorted by
    (p, density):
      rho, p, vmax, replicas;
      J: mean flux over replicas (exact sums, one division), J_sd (sample
        standard deviation over replicas), J_ci95 (half-width of the 95 %
        interval of the mean, Student's t);
      v: mean velocity over replicas;
      J_theory and J_minus_theory where a closed form exists."""
    groups: dict[tuple, list[ReplicaSum]] = {}
    for r in replicas:
        if r.steps <= 0 or r.L <= 0:
            raise ValueError("a replica needs L > 0 and steps > 0")
        groups.setdefault((r.L, r.N, r.p, r.vmax), []).append(r)
    rows = []
    for (L, N, p, vmax), rs in sorted(groups.items(), key=lambda kv: (kv[0][2], Fraction(kv[0][1], kv[0][0]))):
        steps = {r.steps for r in rs}
        if len(steps) != 1:
            raise ValueError("replicas of one point must share the averaging window")
        steps = steps.pop()
        R = len(rs)
        total = sum(r.total_sum_v for r in rs)
        J_exact = Fraction(total, R * L * steps)
        v_exact = Fraction(total, R * N * steps) if N else Fraction(0)
        Js = [Fraction(r.total_sum_v, L * steps) for r in rs]
        if R > 1:
            var = sum((j - J_exact) ** 2 for j in Js) / (R - 1)   # exact sample variance
            sd = math.sqrt(var)
            ci = t_quantile_975(R - 1) * sd / math.sqrt(R)
        else:
            sd, ci = 0.0, float("nan")
        rho = Fraction(N, L)
        row = {"L": L, "N": N, "rho": float(rho), "p": p, "vmax": vmax, "replicas": R, "steps": steps,
               "J": float(J_exact), "J_sd": sd, "J_ci95": ci, "v": float(v_exact)}
        th = theory_flux(rho, p, vmax)
        if th is not None:
            row["J_theory"] = float(th)
            row["J_minus_theory"] = float(J_exact - th) if isinstance(th, Fraction) else float(J_exact) - th
        rows.append(row)
    return rows


def summary(rows: list[dict]) -> dict:
    """Largest |J - theory| over the rows with a closed form, and how many
    of them lie within their 95 % interval (or equal the theory exactly)."""
    th = [r for r in rows if "J_theory" in r]
    within = sum(1 for r in th if r["J_minus_theory"] == 0 or abs(r["J_minus_theory"]) <= r["J_ci95"])
    return {"points": len(rows), "theory_points": len(th),
            "max_abs_J_minus_theory": max((abs(r["J_minus_theory"]) for r in th), default=None),
            "theory_points_within_ci95": within}
