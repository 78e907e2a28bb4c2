"""GPU parity of batched runs (nasch_submit) against the oracle.

A batch mixes every kind of work item (agent warp-tiles, grid spans,
whole-ring agent and grid roads), uneven step counts (including 0), p = 0
and p = 1, wide vmax, a lone car and a full ring.  Every road must equal the
oracle bit for bit, and equal the same road run alone through the
single-road API (the draws are keyed by road id, never by slot or order).
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


MIXED = [
    dict(L=200000, N=9000, vmax=5, p=0.13, seed=3, road_id=11, T=57),            # agent tiles
    dict(L=30000, N=1500, vmax=8, p=0.3, seed=4, road_id=12, T=101),             # agent ring
    dict(L=50000, N=20000, vmax=5, p=0.25, seed=5, road_id=13, T=73),            # grid tiles
    dict(L=5000, N=2500, vmax=3, p=0.5, seed=6, road_id=14, T=90),               # grid ring
    dict(L=40000, N=9000, vmax=20, p=0.1, seed=7, road_id=15, T=33, layout="grid"),   # vmax > 16
    dict(L=60000, N=7000, vmax=5, p=0.0, seed=8, road_id=16, T=40),              # p = 0
    dict(L=60000, N=20000, vmax=5, p=1.0, seed=8, road_id=17, T=40),             # p = 1
    dict(L=1000, N=10, vmax=5, p=0.1, seed=9, road_id=18, T=0),                  # no steps
    dict(L=1000, N=1, vmax=5, p=0.1, seed=9, road_id=19, T=25),                  # a lone car
    dict(L=3000, N=3000, vmax=5, p=0.5, seed=9, road_id=20, T=5),                # full ring
    dict(L=2**31, N=5000, vmax=5, p=0.13, seed=10, road_id=21, T=16),           # wrap at 2^31
    dict(L=9000, N=2100, vmax=127, p=0.2, seed=2, road_id=22, T=12, layout="agent", k=5),
    dict(L=8192 * 3 + 5, N=3000, vmax=5, p=0.2, seed=2, road_id=23, T=30, layout="grid", k=3),
]


def _params(r):
    return {k: r[k] for k in ("L", "N", "vmax", "p", "seed", "road_id", "layout", "k") if k in r}


def oracle_road(r):
    x0 = O.floyd_init(r["L"], r["N"], r["seed"], r["road_id"])
    return O.agent_run(r["L"], x0, np.zeros(r["N"], np.uint8), r["vmax"], r["p"], r["seed"], r["road_id"], 0,
                       r["T"], openmp=True)


def check_road(b, i, r):
    ox, ov, osv, ocr = oracle_road(r)
    sv, cr = b.stats(i)
    assert np.array_equal(sv, osv) and np.array_equal(cr, ocr), (i, "stats")
    assert np.array_equal(b.read_grid(i), O.agent_to_grid(r["L"], ox, ov)), (i, "grid")
    if b.layout(i) == NS.LAYOUT_AGENT:
        x, v = b.read_state(i)
        assert np.array_equal(x, ox) and np.array_equal(v, ov), (i, "agent state")


def test_mixed_batch_matches_oracle():
    with NS.Batch([_params(r) for r in MIXED], [r["T"] for r in MIXED]) as b:
        b.wait()
        inf = b.info()
        assert inf.n_roads == len(MIXED) and inf.super_steps >= 1
        for i, r in enumerate(MIXED):
            check_road(b, i, r)


def test_batch_equals_each_road_alone():
    with NS.Batch([_params(r) for r in MIXED], [r["T"] for r in MIXED]) as b:
        b.wait()
        for i, r in enumerate(MIXED):
            lay = "agent" if b.layout(i) == NS.LAYOUT_AGENT else "grid"
            with NS.Road(r["L"], r["N"], r["vmax"], r["p"], r["seed"], r["road_id"], layout=lay) as alone:
                alone.run(r["T"])
                sv, cr = alone.stats()
                assert np.array_equal(alone.read_grid(), b.read_grid(i)), i
                bsv, bcr = b.stats(i)
                assert np.array_equal(sv, bsv) and np.array_equal(cr, bcr), i


def test_order_and_fusion_depth_do_not_matter():
    rs = [_params(r) for r in MIXED]
    steps = [r["T"] for r in MIXED]
    with NS.Batch(rs, steps) as a:
        a.wait()
        want = [a.read_grid(i) for i in range(len(rs))]
    perm = list(reversed(range(len(rs))))
    rs2 = [dict(rs[i], k=k) for i, k in zip(perm, [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13])]
    with NS.Batch(rs2, [steps[i] for i in perm]) as b:
        b.wait()
        for j, i in enumerate(perm):
            assert np.array_equal(b.read_grid(j), want[i]), i


def test_uneven_ensemble_subset():
    """The 256 smallest-work roads of the seed-7 ensemble, full length, against
    the oracle, and 16 others checked on light-cone windows of cars."""
    rows = WL.uneven_ensemble()
    order = sorted(range(len(rows)), key=lambda i: rows[i]["N"] * rows[i]["T"])
    small = order[:256]
    rng = np.random.default_rng(5)
    mids = [i for i in order[256:] if rows[i]["T"] <= 3000 and rows[i]["N"] > 2048]
    big = list(rng.choice(mids, 16, replace=False))
    pick = small + big
    roads = [WL.road_params(rows[i]) for i in pick]
    steps = [rows[i]["T"] for i in pick]
    with NS.Batch(roads, steps) as b:
        b.wait()
        for j in range(len(small)):
            r = dict(roads[j], T=steps[j])
            check_road(b, j, r)
        for j in range(len(small), len(pick)):
            r = dict(roads[j], T=steps[j])
            x0 = O.floyd_init(r["L"], r["N"], r["seed"], r["road_id"])
            lay = b.layout(j)
            if lay == NS.LAYOUT_AGENT:
                x, v = b.read_state(j)
            else:
                cells = b.read_grid(j)
            for start in rng.integers(0, r["N"], 2):
                M = r["T"] + 40
                idx = (int(start) + np.arange(M)) % r["N"]
                wx, wv = O.agent_segment(r["L"], x0[idx], np.zeros(M, np.uint8), r["vmax"], r["p"], r["seed"],
                                         r["road_id"], 0, r["T"], openmp=True)
                if lay == NS.LAYOUT_AGENT:
                    assert np.array_equal(wx, x[idx[:40]]) and np.array_equal(wv, v[idx[:40]])
                else:
                    assert np.array_equal(cells[wx], wv.astype(np.int8))


def test_fundamental_diagram_subset_matches_oracle():
    """One replica per (density, p) of the sweep, on a shorter road and run."""
    roads = WL.fundamental_diagram_roads(replicas=1, L=20000)
    T = 60
    with NS.Batch(roads, [T] * len(roads)) as b:
        b.wait()
        for i in range(0, len(roads), 5):
            check_road(b, i, dict(roads[i], T=T))


def _invariants(b, i, r):
    """Car count, distinct cells, velocities within vmax, and the statistics'
    length, on a road of the batch."""
    cells = b.read_grid(i)
    occ = cells >= 0
    assert int(occ.sum()) == r["N"], (i, "car count")
    assert int(cells[occ].max(initial=0)) <= r["vmax"], (i, "vmax")
    sv, cr = b.stats(i)
    assert len(sv) == r["T"] and len(cr) == r["T"]
    return cells


@pytest.fixture
def byte_crossover():
    """Automatic layout at the state-byte crossover (agent below density
    0.2, grid above), so a sweep runs in both layouts."""
    prev = NS.get_tuning()
    NS.set_tuning(0.2, 0, 0)
    yield
    NS.set_tuning(*prev)


def test_fundamental_diagram_full_size(byte_crossover):
    """The sweep at full size: one replica per (density, p), L = 10^6, T =
    12000, in the layouts the batch picks at the state-byte crossover.  Every
    road: invariants, and the same cells and statistics when every road is
    forced into the other layout.  Every fourth road: light-cone windows of
    40 cars after the 12000 steps against the oracle run from the same
    start."""
    roads = WL.fundamental_diagram_roads(replicas=1)
    T = WL.FD_T
    with NS.Batch(roads, [T] * len(roads)) as b:
        b.wait()
        layouts = [b.layout(i) for i in range(len(roads))]
        assert NS.LAYOUT_AGENT in layouts and NS.LAYOUT_GRID in layouts
        cells = [_invariants(b, i, dict(r, T=T)) for i, r in enumerate(roads)]
        stats = [b.stats(i) for i in range(len(roads))]
    other = [dict(r, layout="grid" if lay == NS.LAYOUT_AGENT else "agent") for r, lay in zip(roads, layouts)]
    with NS.Batch(other, [T] * len(other)) as b2:
        b2.wait()
        for i in range(len(other)):
            assert np.array_equal(b2.read_grid(i), cells[i]), (i, "layout")
            sv, cr = b2.stats(i)
            assert np.array_equal(sv, stats[i][0]) and np.array_equal(cr, stats[i][1]), (i, "layout stats")
    rng = np.random.default_rng(12)
    for i in range(0, len(roads), 4):
        r = roads[i]
        x0 = O.floyd_init(r["L"], r["N"], r["seed"], r["road_id"])
        M = T + 40
        start = int(rng.integers(0, r["N"]))
        idx = (start + np.arange(M)) % r["N"]
        wx, wv = O.agent_segment(r["L"], x0[idx], np.zeros(M, np.uint8), r["vmax"], r["p"], r["seed"],
                                 r["road_id"], 0, T, openmp=True)
        assert np.array_equal(cells[i][wx], wv.astype(np.int8)), (i, "window")


def test_fundamental_diagram_full_length_roads_match_oracle(byte_crossover):
    """Four roads of the sweep at full size (L = 10^6, T = 12000 steps), one
    per p, at densities next to the critical density 1/(vmax+1) and above
    it, in the layouts the sweep's batch picks (agent below density 0.2, grid
    above): the final state and every step's statistics against the oracle
    run in full from the same Floyd start."""
    picks = [(10, 0), (11, 1), (40, 2), (63, 3)]     # (density index, p index)
    per = len(WL.FD_PS)
    roads = [WL.fundamental_diagram_roads(replicas=1)[i * per + j] for i, j in picks]
    T = WL.FD_T
    with NS.Batch(roads, [T] * len(roads)) as b:
        b.wait()
        layouts = [b.layout(i) for i in range(len(roads))]
        assert NS.LAYOUT_AGENT in layouts and NS.LAYOUT_GRID in layouts
        for i, r in enumerate(roads):
            check_road(b, i, dict(r, T=T))


@pytest.mark.parametrize("layout", ["agent", "grid"])
def test_reference_case_thousand_seeds(layout):
    """The handout's reference case (200 cars on 1000 cells, p = 0.13, vmax =
    5, 1000 steps) for seeds 1..1000, all in one batch, against the oracle."""
    s = WL.REFERENCE_CASE
    roads = [dict(L=s.L, N=s.N, vmax=s.vmax, p=s.p, seed=seed, road_id=0, layout=layout)
             for seed in range(1, 1001)]
    with NS.Batch(roads, [s.T] * len(roads)) as b:
        b.wait()
        for i, r in enumerate(roads):
            check_road(b, i, dict(r, T=s.T))


def test_stats_sum_equals_summed_series_and_oracle():
    """nasch_batch_stats_sum over windows of a road's steps equals the sum
    of the per-step series nasch_batch_stats returns and the sum of the
    oracle's series (the fundamental diagram's time averages come from it)."""
    rs = MIXED[:7]
    with NS.Batch([_params(r) for r in rs], [r["T"] for r in rs]) as b:
        b.wait()
        for i, r in enumerate(rs):
            _, _, osv, ocr = oracle_road(r)
            sv, cr = b.stats(i)
            T = r["T"]
            for first, count in ((0, T), (0, 0), (T // 3, T - T // 3), (1, max(T - 2, 0)), (T - 1, 1)):
                a, c = b.stats_sum(i, first, count)
                assert a == int(sv[first:first + count].sum()) == int(osv[first:first + count].sum()), (i, first)
                assert c == int(cr[first:first + count].sum()) == int(ocr[first:first + count].sum()), (i, first)
        with pytest.raises(NS.NaschError) as e:
            b.stats_sum(0, 1, rs[0]["T"])          # one step past the end
        assert e.value.status == NS.EINVAL


def test_wait_timeout_and_cancel():
    roads = [dict(L=2_000_000, N=200_000, vmax=5, p=0.13, seed=1, road_id=i) for i in range(16)]
    b = NS.Batch(roads, [20000] * len(roads))
    try:
        with pytest.raises(NS.NaschError) as e:
            b.wait(0)
        assert e.value.status == NS.ETIMEOUT
        b.cancel()
        with pytest.raises(NS.NaschError) as e:
            b.wait(120000)
        assert e.value.status == NS.ECANCELED
    finally:
        b.close()


def test_submit_rejects_bad_roads():
    with pytest.raises(NS.NaschError) as e:
        NS.Batch([dict(L=100, N=200)], [10])
    assert e.value.status == NS.EINVAL
    with pytest.raises(NS.NaschError):
        NS.Batch([dict(L=100, N=20)], [-1])


@pytest.fixture
def clean_tuning():
    prev_table = NS.get_tuning_table()
    prev = NS.get_tuning()
    yield
    NS.set_tuning_table(prev_table)
    NS.set_tuning(*prev)


def test_tuned_batch_equals_untuned(clean_tuning):
    """A per-road table that changes every AUTO road's layout, fusion depth
    and grid tile gives the same cells and statistics as the default."""
    rs = [_params(r) for r in MIXED]
    steps = [r["T"] for r in MIXED]
    with NS.Batch(rs, steps) as a:
        a.wait()
        want = [(a.read_grid(i), *a.stats(i)) for i in range(len(rs))]
        lay0 = [a.layout(i) for i in range(len(rs))]
    table = []
    for r, lay in zip(MIXED, lay0):
        flip = "grid" if lay == NS.LAYOUT_AGENT else "agent"
        table.append(dict(L_min=r["L"], L_max=r["L"] + 1, rho_min=0.0, rho_max=1.01, vmax_min=r["vmax"],
                          vmax_max=r["vmax"], draw=-1, layout=flip, k=3 + len(table) % 5, tile=8192))
    NS.set_tuning_table(table)
    with NS.Batch(rs, steps) as b:
        b.wait()
        for i, r in enumerate(MIXED):
            if "layout" not in r:
                assert b.layout(i) != lay0[i], i
            g, sv, cr = want[i]
            assert np.array_equal(b.read_grid(i), g), i
            bsv, bcr = b.stats(i)
            assert np.array_equal(bsv, sv) and np.array_equal(bcr, cr), i


def test_bucket_tuning_is_no_slower_than_the_global_choice(clean_tuning):
    """Two contrasting buckets (short dense roads with vmax 3; long sparse
    roads with vmax 8): the tuned table runs each bucket's batch at least
    0.9 times as fast as the global default (best of three runs each)."""
    from paper_2309_14311_gb300 import autotune as AT
    bs = [dict(L_min=1_000, L_max=10_000, rho_min=0.4, rho_max=1.0001, vmax=3),
          dict(L_min=1_000_000, L_max=10_000_001, rho_min=0.0, rho_max=0.2, vmax=8)]
    res = AT.tune_buckets(bs, steps=64, repeats=1)
    assert len(res["entries"]) == 2
    for b in bs:
        roads = AT.representative_roads(b)
        NS.set_tuning_table([])
        base = max(AT.time_batch(roads, 64) for _ in range(3))
        NS.set_tuning_table(res["entries"])
        tuned = max(AT.time_batch(roads, 64) for _ in range(3))
        assert tuned >= 0.9 * base, (b, tuned, base)


def test_batch_start_states_equal_sequential_floyd():
    """The batch's start states (Floyd's algorithm by one block per road,
    1024 draws at a time) equal the oracle's sequential Floyd: sparse and
    dense roads, a full ring, one car, roads of one and of many groups."""
    shapes = [(1000, 1), (1000, 999), (3000, 3000), (50_000, 1024), (50_000, 1025), (200_000, 150_000),
              (2_000_000, 1_200_000), (10_000_000, 300_000), (2**31, 70_000), (4097, 4096)]
    roads = [dict(L=L, N=N, vmax=5, p=0.1, seed=11 + i, road_id=100 + i, layout="agent")
             for i, (L, N) in enumerate(shapes)]
    with NS.Batch(roads, [0] * len(roads)) as b:
        b.wait()
        for i, r in enumerate(roads):
            x, v = b.read_state(i)
            assert np.array_equal(x, O.floyd_init(r["L"], r["N"], r["seed"], r["road_id"])), shapes[i]
            assert not v.any()
