"""The debug build (-DNASCH_DEBUG) on small cases.

In the debug build every kernel checks, at the points where a wrong value
or index would corrupt the state or memory, that it stays in range; a
failing check sets a bit in a device word (never a trap), and every run is
followed by a check of the whole state on the device.  Here the debug
library runs small roads (L <= 64, and a few larger ones that take the
tiled kernels) in a child process that loads it (NASCH_LIBRARY=debug); all
results must equal the oracle and no check may fire.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
from oracle import oracle as O
from paper_2309_14311_gb300 import nasch as NS
from paper_2309_14311_gb300 import decomp as DC
import torch
assert NS.library_path().endswith("libnasch_debug.so")
NS.load()
cases = []
for L in (1, 2, 7, 16, 33, 64):
    for N in sorted({0, 1, L // 2, L}):
        for vmax, p in ((1, 0.0), (5, 0.3), (5, 1.0)):
            cases.append((L, N, vmax, p, 40, "auto", 0))
cases += [(60_000, 4_000, 5, 0.13, 37, "agent", 16), (60_000, 4_000, 5, 0.13, 37, "grid", 1),
          (60_000, 9_000, 5, 0.25, 37, "grid", 8), (70_000, 20_000, 20, 0.2, 9, "grid", 30)]
for L, N, vmax, p, T, layout, k in cases:
    x0 = O.floyd_init(L, N, 3, 1)
    ox, ov, osv, ocr = O.agent_run(L, x0, np.zeros(N, np.uint8), vmax, p, 3, 1, 0, T)
    with NS.Road(L, N, vmax, p, 3, 1, layout=layout, k=k) as r:
        r.run(T)
        sv, cr = r.stats()
        assert np.array_equal(sv, osv) and np.array_equal(cr, ocr), (L, N, layout)
        assert np.array_equal(r.read_grid(), O.agent_to_grid(L, ox, ov)), (L, N, layout)
roads = [dict(L=c[0], N=c[1], vmax=c[2], p=c[3], seed=3, road_id=1) for c in cases]
with NS.Batch(roads, [c[4] for c in cases]) as b:
    b.wait()
    for i, c in enumerate(cases):
        x0 = O.floyd_init(c[0], c[1], 3, 1)
        ox, ov, osv, ocr = O.agent_run(c[0], x0, np.zeros(c[1], np.uint8), c[2], c[3], 3, 1, 0, c[4])
        assert np.array_equal(b.read_grid(i), O.agent_to_grid(c[0], ox, ov)), ("batch", i)
L, N, vmax, p, k, T = 50_000, 3_000, 5, 0.13, 8, 30
x0 = O.floyd_init(L, N, 3, 1)
segs = DC.segments(L, 3, k, vmax)
bufs = []
for s in segs:
    buf = torch.full((s.W,), -1, dtype=torch.int8)
    j = (x0.astype(np.int64) - s.a) % L
    buf[torch.from_numpy(s.H + j[j < s.owned])] = 0
    bufs.append(buf.cuda())
bufs, _ = DC.run_local(segs, bufs, T, DC.library_step(L, vmax, p, 3, 1))
ox, ov, _, _ = O.agent_run(L, x0, np.zeros(N, np.uint8), vmax, p, 3, 1, 0, T)
got = np.concatenate([b[s.owned_part()].cpu().numpy() for s, b in zip(segs, bufs)])
assert np.array_equal(got, O.agent_to_grid(L, ox, ov)), "segments"
print("debug build ok:", len(cases), "roads")
'''


def test_debug_build_runs_small_cases_without_a_failed_check():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_14311_gb300 import build
    lib = build.build(debug=True)
    assert lib.endswith("libnasch_debug.so")
    env = dict(os.environ, NASCH_LIBRARY="debug", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    p = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    assert "debug build ok" in p.stdout
