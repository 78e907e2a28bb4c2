"""Output while running (nasch_run_output): snapshots of the cells every
`per` steps and the space-time raster, against the oracle's states at the
same steps."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import nasch as NS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    torch.cuda.set_device(0)
    NS.load(build_if_missing=True)


def oracle_states(L, N, vmax, p, seed, road, per, count):
    """Oracle cells after per, 2 per, ..., count * per steps."""
    x = O.floyd_init(L, N, seed, road)
    v = np.zeros(N, np.uint8)
    out = []
    for j in range(count):
        x, v, _, _ = O.agent_run(L, x, v, vmax, p, seed, road, j * per, per, openmp=True)
        out.append((x.copy(), v.copy()))
    return out


@pytest.mark.parametrize("layout,tile,k", [("agent", 512, 8), ("grid", 8192, 1), ("grid", 8192, 4),
                                           ("agent", 0, 4), ("grid", 0, 4)])
def test_snapshots_and_raster_match_oracle(layout, tile, k):
    L, N, vmax, p, seed, road = (50000, 6123, 5, 0.2, 9, 2) if tile else (3000, 700, 5, 0.2, 9, 2)
    per, count, W = 7, 5, 333
    want = oracle_states(L, N, vmax, p, seed, road, per, count)
    snaps = np.zeros((count, L), np.int8)
    rows = np.zeros((count, W), np.uint8)
    with NS.Road(L, N, vmax, p, seed, road, layout=layout, k=k, tile=tile) as r:
        r.run_output(per * count + 3, per, snaps, rows)   # 3 more steps: a partial chunk, no snapshot
        assert r.info().step == per * count + 3
        for j, (x, v) in enumerate(want):
            assert np.array_equal(snaps[j], O.agent_to_grid(L, x, v)), j
            assert np.array_equal(rows[j], O.raster_row(L, x, W)), j
        # the run goes on from the state after the partial chunk
        x, v = want[-1]
        fx, fv, _, _ = O.agent_run(L, x, v, vmax, p, seed, road, per * count, 3, openmp=True)
        assert np.array_equal(r.read_grid(), O.agent_to_grid(L, fx, fv))


def test_ring_of_slots_keeps_the_last_snapshots():
    L, N, vmax, p, seed = 40000, 5000, 5, 0.13, 4
    per, count = 5, 5
    want = oracle_states(L, N, vmax, p, seed, 0, per, count)
    snaps = np.zeros((2, L), np.int8)
    rows = np.zeros((3, 64), np.uint8)
    with NS.Road(L, N, vmax, p, seed, layout="grid", k=1, tile=8192) as r:
        r.run_output(per * count, per, snaps, rows)
    # snapshot j lands in slot j mod 2; j = 4 in slot 0, j = 3 in slot 1
    assert np.array_equal(snaps[0], O.agent_to_grid(L, *want[4]))
    assert np.array_equal(snaps[1], O.agent_to_grid(L, *want[3]))
    # raster row j in slot j mod 3: rows 3, 4, 2
    for slot, j in ((0, 3), (1, 4), (2, 2)):
        assert np.array_equal(rows[slot], O.raster_row(L, want[j][0], 64))


def test_output_off_runs_the_steps():
    L, N = 20000, 3000
    with NS.Road(L, N, 5, 0.3, 1, layout="agent", k=4, tile=512) as r:
        snaps = np.zeros((1, L), np.int8)
        r.run_output(40, 0, snaps, None)            # per = 0: no output
        assert not snaps.any()
        r.run_output(10, 5, None, None)             # no output buffers
        assert r.info().step == 50
        x, v, _, _ = O.agent_run(L, O.floyd_init(L, N, 1, 0), np.zeros(N, np.uint8), 5, 0.3, 1, 0, 0, 50)
        rx, rv = r.read_state()
        assert np.array_equal(rx, x) and np.array_equal(rv, v)


def test_bad_arguments_are_refused():
    with NS.Road(20000, 100, 5, 0.3, 1, layout="grid", k=1, tile=8192) as r:
        lib = NS.load()
        for args in ((-1, 5, None, 0, None, 0, 0), (10, -1, None, 0, None, 0, 0)):
            assert lib.nasch_run_output(r._h, *args) == NS.EINVAL
        rows = np.zeros((2, 8), np.uint8)
        assert lib.nasch_run_output(r._h, 10, 5, None, 0, NS._ptr(rows), 0, 2) == NS.EINVAL       # width 0
        assert lib.nasch_run_output(r._h, 10, 5, None, 0, NS._ptr(rows), 20001, 2) == NS.EINVAL   # width > L
        snaps = np.zeros((1, 20000), np.int8)
        assert lib.nasch_run_output(r._h, 10, 5, NS._ptr(snaps), 0, None, 0, 0) == NS.EINVAL      # no slot
        assert r.info().step == 0
