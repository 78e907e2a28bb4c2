"""The autotuner's choice of the layout crossover density from measured
rates (host logic, no GPU), and (GPU) a tuning run that applies its choice."""
import pytest

from paper_2309_14311_gb300 import autotune as AT


def test_crossover_between_the_last_agent_win_and_the_first_lasting_grid_win():
    d = [0.05, 0.1, 0.2, 0.3, 0.5]
    assert AT.crossover(d, [9, 8, 6, 4, 2], [3, 5, 7, 8, 9]) == pytest.approx(0.15)
    assert AT.crossover(d, [9, 9, 9, 9, 9], [1, 1, 1, 1, 1]) == 1.0
    assert AT.crossover(d, [1, 1, 1, 1, 1], [9, 9, 9, 9, 9]) == 0.0
    # a grid win followed by an agent win does not count
    assert AT.crossover(d, [5, 1, 9, 1, 1], [1, 5, 1, 5, 5]) == pytest.approx(0.25)


def test_crossover_ignores_input_order():
    assert AT.crossover([0.5, 0.05, 0.2], [1, 9, 6], [9, 1, 7]) == pytest.approx(0.125)


@pytest.mark.gpu
def test_tuning_run_applies_its_choice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_14311_gb300 import build
    from paper_2309_14311_gb300 import nasch as NS
    build.build()
    prev = NS.get_tuning()
    res = AT.tune(L=1 << 20, steps=16)
    assert res["k_agent"] in AT.K_CANDIDATES and res["k_grid"] in AT.K_CANDIDATES
    assert 0.0 <= res["rho_star"] <= 1.0
    AT.apply(res)
    rho, ka, kg = NS.get_tuning()
    assert (rho, ka, kg) == (pytest.approx(res["rho_star"]), res["k_agent"], res["k_grid"])
    NS.set_tuning(*prev)


# ---------------------------------------------------------------- per-road table (host lookup; no GPU)
@pytest.fixture
def table_lib():
    from paper_2309_14311_gb300 import build
    from paper_2309_14311_gb300 import nasch as NS
    build.build()
    NS.load()
    prev_table = NS.get_tuning_table()
    prev = NS.get_tuning()
    yield NS
    NS.set_tuning_table(prev_table)
    NS.set_tuning(*prev)


def test_table_lookup_first_match_and_what_it_decides(table_lib):
    NS = table_lib
    NS.set_tuning(1.0, 8, 8)
    NS.set_tuning_table([
        dict(L_min=10_000, L_max=100_000, rho_min=0.0, rho_max=0.5, vmax_min=3, vmax_max=5, draw=-1,
             layout="grid", k=4, tile=8192),
        dict(L_min=10_000, L_max=100_000, rho_min=0.0, rho_max=1.0, vmax_min=0, vmax_max=127, draw=1,
             layout="agent", k=16, tile=0),
    ])
    road = dict(L=50_000, N=10_000, vmax=5, p=0.25)
    assert NS.tuned_choice(road) == (NS.LAYOUT_GRID, 4, 8192)                 # first entry
    assert NS.tuned_choice(dict(road, N=30_000)) == (NS.LAYOUT_AGENT, 16, 256)   # density 0.6: second
    assert NS.tuned_choice(dict(road, vmax=8)) == (NS.LAYOUT_AGENT, 16, 256)     # vmax 8: second
    assert NS.tuned_choice(dict(road, vmax=8, p=0.0)) == (NS.LAYOUT_AGENT, 8, 256)   # p = 0: no entry, global
    assert NS.tuned_choice(dict(road, L=200_000, N=40_000)) == (NS.LAYOUT_AGENT, 8, 256)   # outside every L
    # the road's own choices win over the table
    assert NS.tuned_choice(dict(road, layout="agent")) == (NS.LAYOUT_AGENT, 4, 256)
    assert NS.tuned_choice(dict(road, k=6)) == (NS.LAYOUT_GRID, 6, 8192)
    # whole-ring roads (L <= 8192 grid) report tile 0
    NS.set_tuning_table([dict(L_min=1, L_max=10_000, rho_min=0, rho_max=1, vmax_min=0, vmax_max=127, draw=-1,
                              layout="grid", k=12, tile=0)])
    assert NS.tuned_choice(dict(L=5_000, N=100, vmax=5, p=0.1)) == (NS.LAYOUT_GRID, 12, 0)
    NS.set_tuning_table([])
    assert NS.get_tuning_table() == []
    assert NS.tuned_choice(road) == (NS.LAYOUT_AGENT, 8, 256)


def test_table_rejects_bad_entries(table_lib):
    NS = table_lib
    good = dict(L_min=1, L_max=10, rho_min=0, rho_max=1, vmax_min=0, vmax_max=5, draw=-1, layout="grid", k=4, tile=0)
    NS.set_tuning_table([good])
    for bad in (dict(L_max=1), dict(rho_max=0), dict(vmax_min=6), dict(draw=3), dict(layout=7), dict(k=65),
                dict(tile=1000)):
        with pytest.raises(NS.NaschError) as e:
            NS.set_tuning_table([good, dict(good, **bad)])
        assert e.value.status == NS.EINVAL
    assert len(NS.get_tuning_table()) == 1     # unchanged by the refused tables


def test_buckets_cover_the_ensemble():
    from paper_2309_14311_gb300 import workloads as WL
    bs = AT.buckets()
    assert len(bs) == 4 * 3 * 3
    for r in WL.uneven_ensemble():
        rho = r["N"] / r["L"]
        hits = [b for b in bs if b["L_min"] <= r["L"] < b["L_max"] and b["rho_min"] <= rho < b["rho_max"]
                and b["vmax"] == r["vmax"]]
        assert len(hits) == 1, r
    for b in bs:
        roads = AT.representative_roads(b)
        assert all(b["L_min"] <= x["L"] < b["L_max"] and x["vmax"] == b["vmax"] for x in roads)
        assert 1 <= len(roads) <= 512
