"""Run one road from the handout's parameter file on the GPU:

    python -m paper_2309_14311_gb300 params.ini [--layout agent|grid|auto] [--width W]

Writes, next to the output prefix, the road every `per` steps (and at step
0): `<prefix>-dens.npy` (uint8, 1 where a car is), `<prefix>-velo.npy`
(int8, the car's velocity or -1), `<prefix>-time.npy` (the steps), the
per-step statistics `<prefix>-stats.npy` (sum of velocities, cars passing
cell L-1), and the space-time diagram (Fig. 1: road across, time down,
dark where cars are) as `<prefix>-spacetime.pgm`.  per = 0 writes only the
final state.  The draws are the library's keyed Philox, so a run is the
same whatever the layout or the GPU.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np

from . import nasch as NS
from . import params as P


def write_pgm(path: str, img: np.ndarray) -> None:
    """Binary greyscale image (P5), 0 black .. 255 white."""
    h, w = img.shape
    with open(path, "wb") as f:
        f.write(f"P5\n{w} {h}\n255\n".encode())
        f.write(np.ascontiguousarray(img, dtype=np.uint8).tobytes())


def run(sp: P.SimParams, layout: str = "auto", width: int = 0) -> dict:
    import torch
    torch.cuda.set_device(0)
    NS.load(build_if_missing=True)
    width = min(sp.L, width or 1024)
    per = sp.per
    n = sp.T // per if per > 0 else 0
    snaps = np.empty((n, sp.L), np.int8)
    rows = np.empty((n, width), np.uint8)
    with NS.Road(sp.L, sp.N, sp.vmax, sp.p, sp.seed, 0, layout=layout) as r:
        first = r.read_grid()
        if n:
            r.run_output(n * per, per, snaps, rows)
        if sp.T > n * per:
            r.run(sp.T - n * per)
        last = r.read_grid()
        sv, cr = r.stats()
    cells = np.concatenate([first[None], snaps]) if n else np.stack([first, last])
    times = np.arange(n + 1, dtype=np.int64) * per if n else np.array([0, sp.T], np.int64)
    pre = sp.outputprefix
    np.save(f"{pre}-dens.npy", (cells >= 0).astype(np.uint8))
    np.save(f"{pre}-velo.npy", cells)
    np.save(f"{pre}-time.npy", times)
    np.save(f"{pre}-stats.npy", np.stack([sv, cr]))
    if n:
        write_pgm(f"{pre}-spacetime.pgm", 255 - rows)
    return {"snapshots": int(len(times)), "final": last, "sum_v": sv, "crossings": cr}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("params", help="the parameter file")
    ap.add_argument("--layout", choices=["auto", "agent", "grid"], default="auto")
    ap.add_argument("--width", type=int, default=1024, help="pixels across the space-time diagram")
    args = ap.parse_args(argv)
    sp = P.load(args.params)
    res = run(sp, args.layout, args.width)
    print(f"{sp.T} steps of L={sp.L}, N={sp.N}: {res['snapshots']} snapshots written to {sp.outputprefix}-*.npy")
    return 0


if __name__ == "__main__":
    sys.exit(main())
