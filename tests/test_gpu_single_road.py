"""GPU parity of the single-road kernels against the oracle, through the C ABI.

Positions, velocities and the per-step statistics must be bit-exact (all the
work is integer; the Philox draw is keyed by cell and step, so any tiling,
fusion depth or layout gives the same answer - the assignment's
reproducibility requirement).  Cases cover the tiled and whole-ring kernels,
ragged tails, the ring wrap in the last tile, tiny and full rings, vmax = 0,
p = 0 and p = 1, and the large road at full size.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import nasch as NS
from paper_2309_14311_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_14311_gb300 import build
    build.build()
    NS.load()


def lib_run(L, N, vmax, p, seed, T, road=0, layout="agent", k=0, tile=0, x0=None, v0=None, step0=0,
            chunks=None):
    with NS.Road(L, N, vmax, p, seed, road, layout=layout, k=k, tile=tile) as r:
        if x0 is not None:
            r.set_state(x0, v0, step0)
        for c in (chunks or [T]):
            r.run(c)
        x, v = r.read_state()
        sv, cr = r.stats()
        grid = r.read_grid()
        return x.copy(), v.copy(), sv.copy(), cr.copy(), grid


def oracle_run(L, N, vmax, p, seed, T, road=0, x0=None, v0=None, step0=0):
    if x0 is None:
        x0 = O.floyd_init(L, N, seed, road)
        v0 = np.zeros(N, np.uint8)
    x, v, sv, cr = O.agent_run(L, x0, v0, vmax, p, seed, road, step0, T, openmp=True)
    return x, v, sv, cr


def assert_same(lib, orc, L, layout):
    x, v, sv, cr, grid = lib
    ox, ov, osv, ocr = orc
    assert np.array_equal(sv, osv), "sum_v series differs"
    assert np.array_equal(cr, ocr), "crossings series differs"
    assert np.array_equal(grid, O.agent_to_grid(L, ox, ov)), "grid differs"
    if layout == "agent":
        assert np.array_equal(x, ox) and np.array_equal(v, ov)


def test_device_philox_matches_oracle():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    for seed in (0, 1, 0xDEADBEEF12345678, 2**64 - 1):
        assert np.array_equal(NS.philox_device(ctr, seed), O.philox_many(ctr, seed))


@pytest.mark.parametrize("layout", ["agent", "grid"])
def test_reference_case_many_seeds(layout):
    s = WL.REFERENCE_CASE
    for seed in range(1, 41):
        lib = lib_run(s.L, s.N, s.vmax, s.p, seed, s.T, layout=layout)
        orc = oracle_run(s.L, s.N, s.vmax, s.p, seed, s.T)
        assert_same(lib, orc, s.L, layout)


def test_example_parameter_file_case():
    s = WL.EXAMPLE_PARAMS
    orc = oracle_run(s.L, s.N, s.vmax, s.p, s.seed, s.T)
    for layout in ("agent", "grid"):
        assert_same(lib_run(s.L, s.N, s.vmax, s.p, s.seed, s.T, layout=layout), orc, s.L, layout)
    assert_same(lib_run(s.L, s.N, s.vmax, s.p, s.seed, s.T, layout="agent", tile=512, k=7), orc, s.L, "agent")


AGENT_TILED = [  # (L, N, vmax, p, k, T)
    (100000, 30000, 5, 0.13, 1, 30),
    (100000, 30000, 5, 0.13, 4, 41),
    (100000, 30000, 5, 0.13, 64, 130),
    (50000, 496 * 12, 8, 0.5, 8, 20),          # exactly twelve warp-tiles
    (50000, 496 * 12 + 5, 3, 0.25, 8, 20),     # ragged last tile
    (70001, 9999, 20, 0.3, 5, 33),
    (1000, 7, 5, 0.13, 8, 50),                 # tile holds the ring many times over
    (1000, 1, 9, 0.2, 3, 40),                  # a car alone
    (5000, 5000, 5, 0.5, 4, 10),               # full ring: nothing moves
    (20000, 3000, 0, 0.5, 4, 10),              # vmax = 0
    (20000, 3000, 5, 0.0, 4, 20),              # p = 0
    (20000, 3000, 5, 1.0, 4, 20),              # p = 1
    (2**31, 4000, 5, 0.13, 8, 24),             # wrap arithmetic at L = 2^31
]


@pytest.mark.parametrize("L,N,vmax,p,k,T", AGENT_TILED)
def test_agent_tiled_matches_oracle(L, N, vmax, p, k, T):
    seed = 1000 + L % 97 + N % 13
    orc = oracle_run(L, N, vmax, p, seed, T, road=3)
    lib = lib_run(L, N, vmax, p, seed, T, road=3, layout="agent", k=k, tile=512)
    x, v, sv, cr, _ = lib
    assert np.array_equal(x, orc[0]) and np.array_equal(v, orc[1])
    assert np.array_equal(sv, orc[2]) and np.array_equal(cr, orc[3])


@pytest.mark.parametrize("L,N,vmax,p,k,T", [AGENT_TILED[i] for i in (1, 4, 6, 7, 12)])
def test_agent_small_tile_matches_oracle(L, N, vmax, p, k, T):
    seed = 2000 + L % 89 + N % 7
    orc = oracle_run(L, N, vmax, p, seed, T, road=4)
    x, v, sv, cr, _ = lib_run(L, N, vmax, p, seed, T, road=4, layout="agent", k=k, tile=256)
    assert np.array_equal(x, orc[0]) and np.array_equal(v, orc[1])
    assert np.array_equal(sv, orc[2]) and np.array_equal(cr, orc[3])


GRID_TILED = [  # (L, N, vmax, p, k, T)
    (40000, 8000, 5, 0.13, 1, 30),
    (40000, 8000, 5, 0.13, 8, 37),
    (8192 * 5 + 7, 9000, 5, 0.25, 4, 25),      # ragged last tile
    (60000, 3000, 20, 0.3, 2, 21),             # vmax > 16: gaps across several chunks
    (60000, 600, 127, 0.1, 1, 15),             # largest vmax
    (50000, 30000, 5, 0.5, 16, 40),            # dense, jams
    (50000, 30000, 5, 0.0, 3, 20),
    (50000, 2000, 5, 1.0, 3, 20),
    (33000, 1, 5, 0.2, 6, 30),                 # a car alone
    (100000, 5000, 8, 0.13, 64, 70),
    (70000, 20000, 20, 0.2, 30, 39),           # halo of k steps above 512: block spans, then a shorter last launch
]


@pytest.mark.parametrize("L,N,vmax,p,k,T", GRID_TILED)
def test_grid_tiled_matches_oracle(L, N, vmax, p, k, T):
    seed = 77 + L % 31
    orc = oracle_run(L, N, vmax, p, seed, T, road=5)
    lib = lib_run(L, N, vmax, p, seed, T, road=5, layout="grid", k=k, tile=8192)
    assert_same(lib, orc, L, "grid")


GRID_ONE_STEP = [  # (L, N, vmax, p, T): one step per launch (k = 1)
    (40000, 8000, 5, 0.13, 30),
    (8192 * 5 + 7, 9000, 5, 0.25, 25),         # ragged last tile
    (50000, 30000, 5, 0.5, 40),                # tiles of more than 1024 cars: listed in passes
    (100000, 99000, 3, 0.2, 30),               # nearly full
    (16384, 16384, 5, 0.5, 3),                 # full ring: nothing moves
    (50000, 30000, 5, 0.0, 20),                # p = 0
    (50000, 2000, 5, 1.0, 20),                 # p = 1
    (20000, 3000, 0, 0.5, 10),                 # vmax = 0: no halo
    (60000, 3000, 16, 0.3, 21),                # largest vmax of the one-step kernel
    (60000, 3000, 17, 0.3, 21),                # smallest vmax past it
    (33000, 1, 5, 0.2, 30),                    # a car alone
    (2**31, 4000, 5, 0.13, 24),                # wrap arithmetic at L = 2^31
]


@pytest.mark.parametrize("L,N,vmax,p,T", GRID_ONE_STEP)
def test_grid_one_step_matches_oracle(L, N, vmax, p, T):
    seed = 91 + L % 37
    orc = oracle_run(L, N, vmax, p, seed, T, road=6)
    lib = lib_run(L, N, vmax, p, seed, T, road=6, layout="grid", k=1, tile=8192)
    assert_same(lib, orc, L, "grid")


@pytest.mark.parametrize("layout,k", [("agent", 8), ("grid", 1), ("grid", 4)])
def test_statistics_after_a_reset_and_growth(layout, k):
    """The per-step series' slots are cleared once, not per call: after
    set_state resets the series, slots that held the earlier steps are
    cleared before reuse (runs below, across and past the old high mark),
    and a series that outgrows its buffer keeps what it held."""
    L, N, vmax, p, seed, road = 30000, 3000, 5, 0.3, 12, 4
    x0 = O.floyd_init(L, N, seed, road)
    v0 = np.zeros(N, np.uint8)
    with NS.Road(L, N, vmax, p, seed, road, layout=layout, k=k, tile=8192 if layout == "grid" else 512) as r:
        r.run(700)
        r.set_state(x0, v0, 0)
        for steps in (5, 300, 1500, 1):
            r.run(steps)
        sv, cr = r.stats()
    _, _, osv, ocr = O.agent_run(L, x0, v0, vmax, p, seed, road, 0, 1806)
    assert len(sv) == 1806
    assert np.array_equal(sv, osv) and np.array_equal(cr, ocr)


def test_grid_one_step_many_tiles_per_warp_mixed_density():
    """The one-step kernel over enough tiles that every warp steps many in
    turn (its copies run ahead of the tile it steps), with dense tiles
    (listed and stepped in passes) and sparse ones along the same ring, and
    the ring's first and last tiles loaded across the wrap point."""
    L = 2**26
    rng = np.random.default_rng(77)
    occ = np.concatenate([rng.random(L // 4) < 0.03, rng.random(L // 4) < 0.5,
                          rng.random(L // 4) < 0.2, rng.random(L - 3 * (L // 4)) < 0.9])
    x = np.flatnonzero(occ).astype(np.int32)
    v = rng.integers(0, 6, x.size).astype(np.uint8)
    cells = np.full(L, -1, np.int8)
    cells[x] = v.astype(np.int8)
    orc, osv, ocr = O.grid_run(cells, 5, 0.2, 3, 9, 100, 6, openmp=True)
    with NS.Road(L, x.size, 5, 0.2, 3, 9, layout="grid", k=1) as r:
        r.set_state(x, v, 100)
        r.run(6)
        sv, cr = r.stats()
        assert np.array_equal(r.read_grid(), orc)
    assert np.array_equal(sv, osv) and np.array_equal(cr, ocr)


@pytest.mark.parametrize("L,N,vmax,p,T", [(200, 50, 5, 0.13, 300), (3, 2, 127, 0.5, 50), (1, 1, 3, 0.5, 5),
                                          (32768, 4000, 20, 0.3, 40), (8192, 8192, 5, 0.5, 3),
                                          (9000, 8192, 2, 0.2, 60), (500, 0, 5, 0.5, 10)])
def test_whole_ring_kernels(L, N, vmax, p, T):
    orc = oracle_run(L, N, vmax, p, 5, T, road=1)
    for layout in ("agent", "grid"):
        assert_same(lib_run(L, N, vmax, p, 5, T, road=1, layout=layout), orc, L, layout)


def test_layout_and_fusion_depth_independence():
    """Same road, every launch configuration: identical results."""
    L, N, vmax, p, T, seed = 50000, 6000, 5, 0.2, 96, 9
    want = lib_run(L, N, vmax, p, seed, T, layout="agent", k=1, tile=512)
    for k in (2, 3, 4, 8, 16, 32, 64):
        got = lib_run(L, N, vmax, p, seed, T, layout="agent", k=k, tile=512)
        for a, b in zip(want, got):
            assert np.array_equal(a, b), k
    for k in (1, 2, 5, 8, 13, 64):
        got = lib_run(L, N, vmax, p, seed, T, layout="grid", k=k, tile=8192)
        for a, b in zip(want[2:], got[2:]):
            assert np.array_equal(a, b), k
    # launches split at odd places
    got = lib_run(L, N, vmax, p, seed, T, layout="agent", k=8, tile=512, chunks=[1, 7, 30, 58])
    for a, b in zip(want, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("layout,tile", [("agent", 0), ("agent", 512), ("grid", 0), ("grid", 8192)])
def test_resume_from_state_is_bit_exact(layout, tile):
    L, N, vmax, p, seed = 40000, 5000, 5, 0.13, 21
    T1, T2 = 37, 45
    full = lib_run(L, N, vmax, p, seed, T1 + T2, layout=layout, tile=tile)
    with NS.Road(L, N, vmax, p, seed, layout=layout, tile=tile) as r:
        r.run(T1)
        x, v = r.read_state()
        x, v = x.copy(), v.copy()
    res = lib_run(L, N, vmax, p, seed, T2, layout=layout, tile=tile, x0=x, v0=v, step0=T1)
    assert np.array_equal(res[4], full[4])
    assert np.array_equal(res[2], full[2][T1:]) and np.array_equal(res[3], full[3][T1:])


def test_set_state_rejects_bad_states():
    """Bad states are refused (checked on the device) and leave the road as
    it was."""
    with NS.Road(100, 3, 5, 0.1, 1, layout="agent") as r:
        x0, v0 = (a.copy() for a in r.read_state())
        for x, v, msg in [([1, 1, 5], [0, 0, 0], "two cars on cell 1"), ([1, 5, 200], [0, 0, 0], "x[2]=200"),
                          ([1, 5, 9], [0, 6, 0], "v[1]=6"), ([5, 1, 9], [0, 0, 0], "cyclic order"),
                          ([-3, 5, 9], [0, 0, 0], "x[0]=-3"), ([9, 5, 9], [0, 0, 0], "two cars on cell 9")]:
            with pytest.raises(NS.NaschError) as e:
                r.set_state(np.array(x), np.array(v), 0)
            assert e.value.status == NS.EINVAL and msg in str(e.value), (x, v, str(e.value))
            x1, v1 = r.read_state()
            assert np.array_equal(x1, x0) and np.array_equal(v1, v0)
        with pytest.raises(NS.NaschError):
            r.set_state(np.array([1, 2]), np.array([0, 0]), 0)   # wrong N
        r.set_state(np.array([9, 1, 5]), np.array([1, 2, 3]), 0)   # rotation of sorted: fine
        with pytest.raises(NS.NaschError):
            r.stats(0, 5)   # nothing run yet


def test_grid_set_state_checks():
    """A grid road takes the cars in any order; a cell shared by two cars
    that are not neighbours in the array is found by counting the occupied
    cells after the scatter.  Refused states leave the road as it was."""
    with NS.Road(100, 4, 5, 0.1, 1, layout="grid") as r:
        before = r.read_grid().copy()
        for x, v, msg in [([1, 5, 9, 5], [0, 0, 0, 0], "two cars on cell 5"),
                          ([3, 3, 7, 9], [0, 0, 0, 0], "two cars on cell 3"),
                          ([2, 50, 100, 7], [0, 0, 0, 0], "x[2]=100"),
                          ([1, 5, 9, 20], [0, 6, 0, 0], "v[1]=6")]:
            with pytest.raises(NS.NaschError) as e:
                r.set_state(np.array(x, np.int32), np.array(v, np.uint8), 0)
            assert e.value.status == NS.EINVAL and msg in str(e.value), (x, str(e.value))
            assert np.array_equal(r.read_grid(), before)
        r.set_state(np.array([9, 1, 5, 20], np.int32), np.array([1, 2, 3, 0], np.uint8), 7)
        want = np.full(100, -1, np.int8)
        want[[9, 1, 5, 20]] = [1, 2, 3, 0]
        assert np.array_equal(r.read_grid(), want)
        r.run(3)
        orc = O.grid_run(want, 5, 0.1, 1, 0, 7, 3)
        assert np.array_equal(r.read_grid(), orc[0])


@pytest.fixture(scope="module")
def large_init():
    s = WL.LARGE_ROAD
    return O.floyd_init(s.L, s.N, s.seed, s.road_id)


def test_large_road_full_size(large_init):
    """The large road at full size (2^31 cells, 2^27 cars) in the launch
    configuration the benchmark times: the start state equals the oracle's,
    the first 100 steps equal the oracle's in full (state and per-step
    statistics), the grid layout (one step per launch, and fused) equals
    the agent layout after 100 steps,
    after 10^4 steps sampled windows of cars equal the oracle's
    light-cone evolution of the same cars from the start, and the fused
    grid layout equals the agent layout after all 10^4 steps."""
    s = WL.LARGE_ROAD
    x0 = large_init
    T0 = 100
    with NS.Road(s.L, s.N, s.vmax, s.p, s.seed, layout="agent", k=WL.LARGE_ROAD_K["agent"]) as r:
        x, v = r.read_state()
        assert np.array_equal(x, x0) and not v.any()
        r.run(T0)
        xa, va = r.read_state()
        xa, va = xa.copy(), va.copy()
        sva, cra = r.stats()
        ox, ov, osv, ocr = O.agent_run(s.L, x0, np.zeros(s.N, np.uint8), s.vmax, s.p, s.seed, 0, 0, T0,
                                       openmp=True)
        assert np.array_equal(sva, osv) and np.array_equal(cra, ocr)
        assert np.array_equal(xa, ox) and np.array_equal(va, ov)
        del ox, ov
        r.run(s.T - T0)
        xT, vT = r.read_state()
        xT, vT = xT.copy(), vT.copy()
        svT, _ = r.stats()
        assert len(svT) == s.T
    # the grid layout in both launch configurations the benchmark times:
    # one step per launch (the one-step list kernel) and the fused depth
    order = np.argsort(xa, kind="stable")
    for kg in (1, WL.LARGE_ROAD_K["grid"]):
        with NS.Road(s.L, s.N, s.vmax, s.p, s.seed, layout="grid", k=kg) as g:
            g.run(T0)
            svg, crg = g.stats()
            assert np.array_equal(svg, sva) and np.array_equal(crg, cra), kg
            xg, vg = g.read_state()   # cars in cell order
            assert np.array_equal(xg, xa[order]) and np.array_equal(vg, va[order]), kg
            del xg, vg
    # sampled light-cone windows over the full 10^4 steps
    rng = np.random.default_rng(2309)
    M = s.T + 48
    for start in list(rng.integers(0, s.N, 5)) + [s.N - 20]:
        idx = (int(start) + np.arange(M)) % s.N
        wx, wv = O.agent_segment(s.L, x0[idx], np.zeros(M, np.uint8), s.vmax, s.p, s.seed, 0, 0, s.T,
                                 openmp=True)
        assert np.array_equal(wx, xT[idx[:M - s.T]]), start
        assert np.array_equal(wv, vT[idx[:M - s.T]]), start
    # the grid layout (fused) over all 10^4 steps equals the agent layout at T
    with NS.Road(s.L, s.N, s.vmax, s.p, s.seed, layout="grid", k=WL.LARGE_ROAD_K["grid"]) as g:
        g.run(s.T)
        svg, _ = g.stats()
        assert np.array_equal(svg, svT)
        xg, vg = g.read_state()   # cars in cell order
        order = np.argsort(xT, kind="stable")
        assert np.array_equal(xg, xT[order]) and np.array_equal(vg, vT[order])
