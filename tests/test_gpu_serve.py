"""GPU tests of the serving loop (continuous batching under a memory budget).

Requests arriving while others run are admitted into the same launches; each
request's per-step statistics and final state must equal the oracle run of
the same road from its Floyd start and the same road run alone through the
single-road API (bit-exact; its draws are keyed by its own seed and road
id).  The budget bounds what is resident; requests that can never fit are
refused; cancelled requests report so.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import nasch as NS
from paper_2309_14311_gb300 import serve as SV
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


def mixed_requests(n, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        L = int(rng.choice([900, 5000, 20000, 70000, 300000]))
        rho = float(rng.uniform(0.03, 0.7))
        N = max(1, min(L, int(rho * L)))
        reqs.append(dict(L=L, N=N, vmax=int(rng.choice([3, 5, 8, 20])), p=float(rng.choice([0.0, 0.13, 0.4, 1.0])),
                         seed=int(rng.integers(1, 1000)), road_id=1000 + i, T=int(rng.integers(0, 120))))
    return reqs


def alone(r):
    rho_star = NS.get_tuning()[0]   # the server's automatic layout choice
    lay = "agent" if r["N"] < rho_star * r["L"] else "grid"
    with NS.Road(r["L"], r["N"], r["vmax"], r["p"], r["seed"], r["road_id"], layout=lay) as road:
        road.run(r["T"])
        sv, cr = road.stats()
        x, v = road.read_state()   # agent: car order; grid: cell order (the server returns the same)
        return sv.copy(), cr.copy(), x.copy(), v.copy()


def oracle_request(r):
    """The request's road run by the oracle: Floyd start of (seed, road id),
    v = 0, T steps.  Returns the per-step series and the final cells."""
    x0 = O.floyd_init(r["L"], r["N"], r["seed"], r["road_id"])
    ox, ov, osv, ocr = O.agent_run(r["L"], x0, np.zeros(r["N"], np.uint8), r["vmax"], r["p"], r["seed"],
                                   r["road_id"], 0, r["T"], openmp=True)
    return osv, ocr, O.agent_to_grid(r["L"], ox, ov)


def test_requests_in_the_mix_equal_oracle_and_alone():
    reqs = mixed_requests(48)
    with NS.Server(memory_budget=1 << 30, steps_per_tick=4, max_resident=16, keep_state=True) as srv:
        # submit in waves while earlier requests are running
        for wave in range(4):
            for i in range(wave * 12, wave * 12 + 12):
                srv.submit(WL.road_params(reqs[i]), reqs[i]["T"], i)
            for _ in range(3):
                srv.step()
        srv.drain(600000)
        results = {r["request_id"]: r for r in srv.poll()}
        assert sorted(results) == list(range(len(reqs)))
        for i, r in enumerate(reqs):
            assert results[i]["status"] == NS.OK
            sv, cr, x, v = srv.result(i, with_state=True)
            osv, ocr, ocells = oracle_request(r)
            assert np.array_equal(sv, osv) and np.array_equal(cr, ocr), (i, "series against the oracle")
            assert np.array_equal(O.agent_to_grid(r["L"], x, v), ocells), (i, "state against the oracle")
            asv, acr, ax, av = alone(r)
            assert np.array_equal(sv, asv) and np.array_equal(cr, acr), i
            assert np.array_equal(x, ax) and np.array_equal(v, av), i
        inf = srv.info()
        assert inf.resident == 0 and inf.queued == 0 and inf.bytes_in_use == 0


def test_budget_bounds_residency_and_oversize_is_refused():
    # each request: agent N=400k -> 2*(1.6 MB + 0.4 MB) + stats, about 4 MB; budget 10 MB
    road = dict(L=4_000_000, N=400_000, vmax=5, p=0.13, seed=1)
    with NS.Server(memory_budget=10 << 20, steps_per_tick=2, max_resident=64) as srv:
        for i in range(6):
            srv.submit(dict(road, road_id=i), 20, i)
        peak = 0
        while srv.step() > 0:
            peak = max(peak, srv.info().resident)
        srv.drain(600000)
        assert 1 <= peak <= 2
        assert len(srv.poll()) == 6
        with pytest.raises(NS.NaschError) as e:
            srv.submit(dict(L=2**31, N=2**20, vmax=5, p=0.1, seed=1, road_id=99), 10, 99)
        assert e.value.status == NS.ENOMEM


def test_cancel_queued_and_running():
    road = dict(L=2_000_000, N=100_000, vmax=5, p=0.13, seed=3)
    with NS.Server(memory_budget=1 << 30, steps_per_tick=2, max_resident=1) as srv:
        srv.submit(dict(road, road_id=1), 200_000, 1)   # long, occupies the only slot
        srv.submit(dict(road, road_id=2), 50, 2)        # waits in the queue
        srv.step()
        srv.cancel(2)
        srv.cancel(1)
        srv.drain(600000)
        res = {r["request_id"]: r for r in srv.poll()}
        assert res[1]["status"] == NS.ECANCELED and res[2]["status"] == NS.ECANCELED


def test_poisson_driver_small_stream_matches_oracle():
    """The smallest requests of the seed-11 stream, served by the Poisson
    driver; every served result equals the oracle run of its road."""
    rows = [r for r in WL.request_stream() if r["N"] * r["T"] < 3e7][:40]
    checked = []

    def check(srv, res):
        i = res["request_id"]
        assert res["status"] == NS.OK, i
        r = dict(WL.road_params(rows[i]), T=rows[i]["T"])
        sv, cr, x, v = srv.result(i, with_state=True)
        osv, ocr, ocells = oracle_request(r)
        assert np.array_equal(sv, osv) and np.array_equal(cr, ocr), (i, "series")
        assert np.array_equal(O.agent_to_grid(r["L"], x, v), ocells), (i, "state")
        checked.append(i)

    out = SV.run_poisson(rows, rate=200.0, memory_budget=2 << 30, steps_per_tick=8, keep_state=True,
                         on_result=check)
    assert out["completed"] == len(rows)
    assert sorted(checked) == list(range(len(rows)))
    assert out["latency_p99_s"] >= out["latency_p50_s"] > 0


def test_series_stream_while_requests_run():
    """Streamed per-step series: chunks of a running request arrive before it
    finishes, in step order; put together they equal the request's final
    series and the oracle's, for a long and a short request and a request
    with no steps."""
    reqs = [dict(L=1_000_000, N=120_000, vmax=5, p=0.13, seed=4, road_id=70, T=3000),
            dict(L=40_000, N=9_000, vmax=8, p=0.3, seed=5, road_id=71, T=200),
            dict(L=5_000, N=100, vmax=5, p=0.2, seed=6, road_id=72, T=0)]
    got = {i: [] for i in range(len(reqs))}
    early = set()
    finished = set()
    with NS.Server(memory_budget=1 << 30, steps_per_tick=2, max_steps_per_tick=2, target_tick_ms=0,
                   ticks_in_flight=2) as srv:
        for i, r in enumerate(reqs):
            srv.submit(WL.road_params(r), r["T"], i)
        pending = 1
        while pending or len(finished) < len(reqs):
            pending = srv.step()
            for rid, first, sv, cr in srv.poll_series(cap_chunks=64, cap_steps=1 << 16):
                if rid not in finished:
                    early.add(rid)
                got[rid].append((first, sv, cr))
            finished |= {res["request_id"] for res in srv.poll()}
        for rid, first, sv, cr in srv.poll_series():
            got[rid].append((first, sv, cr))
        assert srv.poll_series() == []
        for i, r in enumerate(reqs):
            firsts = [c[0] for c in got[i]]
            lens = [len(c[1]) for c in got[i]]
            assert firsts == list(np.cumsum([0] + lens))[:-1], (i, "chunks in step order")
            sv = np.concatenate([c[1] for c in got[i]]) if got[i] else np.zeros(0, np.uint64)
            cr = np.concatenate([c[2] for c in got[i]]) if got[i] else np.zeros(0, np.uint64)
            fsv, fcr = srv.result(i)
            osv, ocr, _ = oracle_request(r)
            assert np.array_equal(sv, fsv) and np.array_equal(cr, fcr), (i, "streamed = final")
            assert np.array_equal(sv, osv) and np.array_equal(cr, ocr), (i, "streamed = oracle")
        assert 0 in early, "the long request's first chunk came only after it finished"
        assert len(got[0]) > 2


def test_tick_grows_when_few_roads_are_resident():
    """With one small road resident, a tick runs more launches than
    steps_per_tick (up to max_steps_per_tick) to reach its GPU-time target;
    the result is unchanged."""
    r = dict(L=200_000, N=20_000, vmax=5, p=0.13, seed=9, road_id=80, T=20_000)
    with NS.Server(memory_budget=1 << 30, steps_per_tick=2, max_steps_per_tick=64, target_tick_ms=5.0) as srv:
        srv.submit(WL.road_params(r), r["T"], 0)
        most = 0
        while srv.step():
            most = max(most, srv.info().last_tick_super_steps)
        srv.drain(600000)
        assert 2 < most <= 64
        assert srv.info().gpu_busy_seconds > 0
        (res,) = srv.poll()
        sv, cr = srv.result(0)
        osv, ocr, _ = oracle_request(r)
        assert np.array_equal(sv, osv) and np.array_equal(cr, ocr)



def test_series_stream_with_small_caps_and_release():
    """poll_series with a step cap smaller than what is ready returns the
    first part and keeps the rest for the next call; chunks of several
    requests share one call; a released request's remaining series is
    dropped."""
    reqs = [dict(L=100_000, N=8_000, vmax=5, p=0.2, seed=21 + i, road_id=90 + i, T=700) for i in range(3)]
    with NS.Server(memory_budget=1 << 30, steps_per_tick=4, max_steps_per_tick=4, target_tick_ms=0) as srv:
        for i, r in enumerate(reqs):
            srv.submit(WL.road_params(r), r["T"], i)
        srv.drain(600000)
        done = {res["request_id"] for res in srv.poll()}
        assert done == {0, 1, 2}
        got = {0: [], 1: []}
        while True:
            chunks = srv.poll_series(cap_chunks=2, cap_steps=150)   # at most 150 steps, 2 chunks per call
            if not chunks:
                break
            assert len(chunks) <= 2 and sum(len(c[2]) for c in chunks) <= 150
            for rid, first, sv, cr in chunks:
                if rid == 2:
                    continue
                got[rid].append((first, sv, cr))
            if 2 in {c[0] for c in chunks}:
                srv.release(2)                                      # the rest of request 2 is dropped
        for i in (0, 1):
            firsts = [c[0] for c in got[i]]
            sv = np.concatenate([c[1] for c in got[i]])
            cr = np.concatenate([c[2] for c in got[i]])
            assert firsts == list(np.cumsum([0] + [len(c[1]) for c in got[i]]))[:-1]
            fsv, fcr = srv.result(i)
            assert np.array_equal(sv, fsv) and np.array_equal(cr, fcr), i
        with pytest.raises((NS.NaschError, KeyError)):   # the request is gone
            srv.result(2)
