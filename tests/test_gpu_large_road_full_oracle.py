"""The large road (2^31 cells, 2^27 cars, density 1/16, vmax 5, p 0.13,
seed 1) over all 10^4 steps against the OpenMP oracle, in full: the final
agent state, the whole per-step series of velocity sums and crossings, and
the fused grid layout's final cells.

About 1.3e12 vehicle-updates of oracle work (close to half an hour on 16
cores), so it runs only when NASCH_FULL_ORACLE=1 is set; the regular GPU
tests check the same road on its first 100 steps in full and on light-cone
windows over the 10^4 steps.
"""
import os
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import nasch as NS
from paper_2309_14311_gb300 import workloads as WL

pytestmark = [
    pytest.mark.gpu,
    pytest.mark.skipif(os.environ.get("NASCH_FULL_ORACLE") != "1",
                       reason="half an hour of oracle time: set NASCH_FULL_ORACLE=1"),
]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_14311_gb300 import build
    build.build()
    NS.load()


def test_large_road_all_steps_against_the_oracle():
    s = WL.LARGE_ROAD
    x0 = O.floyd_init(s.L, s.N, s.seed, s.road_id)
    with NS.Road(s.L, s.N, s.vmax, s.p, s.seed, s.road_id, layout="agent", k=WL.LARGE_ROAD_K["agent"]) as r:
        r.run(s.T)
        x, v = r.read_state()
        x, v = x.copy(), v.copy()
        sv, cr = r.stats()
    with NS.Road(s.L, s.N, s.vmax, s.p, s.seed, s.road_id, layout="grid", k=WL.LARGE_ROAD_K["grid"]) as g:
        g.run(s.T)
        cells = g.read_grid()
    t0 = time.perf_counter()
    ox, ov, osv, ocr = O.agent_run(s.L, x0, np.zeros(s.N, np.uint8), s.vmax, s.p, s.seed, s.road_id, 0, s.T, openmp=True)
    print(f"oracle: {s.N * s.T / (time.perf_counter() - t0):.3e} vehicle-updates/s")
    assert np.array_equal(sv, osv) and np.array_equal(cr, ocr)
    assert np.array_equal(x, ox) and np.array_equal(v, ov)
    want = np.full(s.L, -1, np.int8)
    want[ox] = ov.astype(np.int8)
    del ox, ov
    assert np.array_equal(cells, want)
    print(f"all {s.T} steps equal; sum of velocities over the run {int(osv.sum())}, crossings {int(ocr.sum())}")
