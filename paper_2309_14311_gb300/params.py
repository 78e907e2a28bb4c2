"""The handout's parameter file (Handout, starter code: a plain-text file of
`key = value` lines giving L, T, N, p, vmax, seed, outputprefix and per)."""
from __future__ import annotations

from dataclasses import dataclass

KEYS = ("L", "T", "N", "p", "vmax", "seed", "outputprefix", "per")


@dataclass
class SimParams:
    L: int
    T: int
    N: int
    p: float
    vmax: int
    seed: int
    outputprefix: str
    per: int


def parse(text: str) -> SimParams:
    """Parse `key = value` lines (blank lines and text after '#' ignored;
    string values may be quoted).  Every key must appear exactly once."""
    seen: dict[str, str] = {}
    for n, raw in enumerate(text.splitlines(), 1):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        if "=" not in line:
            raise ValueError(f"line {n}: expected 'key = value', got {raw!r}")
        k, v = (t.strip() for t in line.split("=", 1))
        if k not in KEYS:
            raise ValueError(f"line {n}: unknown key {k!r} (known: {', '.join(KEYS)})")
        if k in seen:
            raise ValueError(f"line {n}: {k} given twice")
        seen[k] = v
    missing = [k for k in KEYS if k not in seen]
    if missing:
        raise ValueError(f"missing keys: {', '.join(missing)}")
    prefix = seen["outputprefix"]
    if len(prefix) >= 2 and prefix[0] == prefix[-1] and prefix[0] in "\"'":
        prefix = prefix[1:-1]
    sp = SimParams(L=int(seen["L"]), T=int(seen["T"]), N=int(seen["N"]), p=float(seen["p"]),
                   vmax=int(seen["vmax"]), seed=int(seen["seed"]), outputprefix=prefix, per=int(seen["per"]))
    if sp.L < 1 or not 0 <= sp.N <= sp.L or sp.T < 0 or sp.per < 0 or not 0 <= sp.vmax <= 127 or not 0 <= sp.p <= 1:
        raise ValueError(f"parameters out of range: {sp}")
    return sp


def load(path: str) -> SimParams:
    with open(path) as f:
        return parse(f.read())
