"""Reader for the hand-worked fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    """Parse `key = value` lines; values are int lists, ints or floats."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, val = (s.strip() for s in line.split("=", 1))
            toks = val.split()
            if k in ("p", "alpha", "beta"):
                out[k] = float(toks[0])
            elif k in ("x", "v", "row") or k.startswith(("x@", "v@")):
                out[k] = [int(t) for t in toks]
            else:
                out[k] = int(toks[0])
    return out


def steps(fx):
    """Step indices t for which the fixture gives x@t."""
    return sorted(int(k[2:]) for k in fx if k.startswith("x@"))


ALL = sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt") and f.startswith(("step_", "single_", "full_")))
