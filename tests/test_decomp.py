"""Multi-rank paths on CPU: the 1-D domain decomposition of one ring road
(decomp.py) and the road-range partition of batches and request streams
(partition.py).

The decomposition's halo exchange is exercised with every rank in one
process and with 2 and 3 gloo ranks exchanging by point-to-point messages;
each rank steps its buffer with the oracle's segment form (cells of a window
after T steps, exact away from the window's edges), and the owned cells put
together must equal the oracle's run of the whole ring.  The partition's
ranks run their road ranges with the oracle; the union of their results,
keyed by road, must equal the single-rank results.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2309_14311_gb300 import decomp as DC
from paper_2309_14311_gb300 import partition as PT


def oracle_step(L, vmax, p, seed, road):
    """step_fn over numpy or torch CPU buffers: the oracle's window run."""
    def step(seg, buf_in, buf_out, k, step0, rank):
        cells = buf_in.numpy() if hasattr(buf_in, "numpy") else buf_in
        mid = O.grid_segment(L, cells, seg.first_buffer_cell, vmax, p, seed, road, step0, k)
        m = k * vmax
        owned = mid[seg.H - m: seg.H - m + seg.owned]
        if hasattr(buf_out, "numpy"):
            buf_out[seg.owned_part()] = torch.from_numpy(owned.copy())
        else:
            buf_out[seg.owned_part()] = owned
        return None
    return step


def start_ring(L, N, seed, road):
    return O.agent_to_grid(L, O.floyd_init(L, N, seed, road), np.zeros(N, np.uint8))


def fill(seg, ring):
    """A rank's buffer from the whole ring (the halos are overwritten by the
    first exchange)."""
    return ring[np.array(seg.ring_cells())].copy()


@pytest.mark.parametrize("L,world", [(1000, 1), (1000, 3), (1001, 7), (97, 4), (2**31, 5)])
def test_owned_ranges_cover_the_ring(L, world):
    rs = [DC.owned_range(L, world, r) for r in range(world)]
    assert rs[0][0] == 0 and rs[-1][1] == L
    assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
    sizes = [b - a for a, b in rs]
    assert max(sizes) - min(sizes) <= 1


def test_segment_geometry_and_limits():
    s = DC.RingSegment(L=1000, world=3, rank=1, k=4, vmax=5)
    assert s.H == 32 and (s.a, s.b) == (333, 666) and s.W == 333 + 64
    assert s.left == 0 and s.right == 2 and s.first_buffer_cell == 301
    assert s.ring_cells()[:2] == [301, 302] and s.ring_cells()[-1] == 697
    s0 = DC.RingSegment(L=1000, world=3, rank=0, k=4, vmax=5)
    assert s0.first_buffer_cell == 1000 - 32 and s0.left == 2
    with pytest.raises(ValueError):
        DC.RingSegment(L=100, world=4, rank=0, k=8, vmax=5)    # owns 25 cells, halo 48


@pytest.mark.parametrize("L,N,vmax,p,k,world,T", [
    (3000, 400, 5, 0.13, 4, 1, 37),
    (3000, 400, 5, 0.13, 4, 2, 37),
    (3001, 1500, 5, 0.5, 3, 3, 20),
    (5000, 900, 8, 0.25, 2, 4, 25),
    (2000, 300, 5, 0.0, 6, 3, 30),
    (2000, 1200, 3, 1.0, 5, 2, 17),
])
def test_local_decomposition_equals_whole_ring(L, N, vmax, p, k, world, T):
    seed, road = 3, 11
    ring = start_ring(L, N, seed, road)
    want, _, _ = O.grid_run(ring, vmax, p, seed, road, 0, T)
    segs = DC.segments(L, world, k, vmax)
    bufs = [fill(s, ring) for s in segs]
    bufs, _ = DC.run_local(segs, bufs, T, oracle_step(L, vmax, p, seed, road))
    got = np.concatenate([b[s.owned_part()] for s, b in zip(segs, bufs)])
    assert np.array_equal(got, want)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _decomp_rank(rank, world, port, case, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, N, vmax, p, k, T, seed, road = case
    ring = start_ring(L, N, seed, road)
    seg = DC.RingSegment(L, world, rank, k, vmax)
    buf = torch.from_numpy(fill(seg, ring))
    buf[seg.left_halo()] = -7          # stale halos: the exchange must replace them
    buf[seg.right_halo()] = -7
    buf, _ = DC.run_rank(seg, buf, T, oracle_step(L, vmax, p, seed, road), dist)
    out[rank] = buf[seg.owned_part()].numpy().tobytes()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_halos(world):
    case = (4000, 700, 5, 0.13, 4, 29, 5, 2)
    L, N, vmax, p, k, T, seed, road = case
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_decomp_rank, args=(r, world, port, case, out)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(180)
            assert pr.exitcode == 0
        parts = [np.frombuffer(out[r], dtype=np.int8) for r in range(world)]
    want, _, _ = O.grid_run(start_ring(L, N, seed, road), vmax, p, seed, road, 0, T)
    assert np.array_equal(np.concatenate(parts), want)


# ---------------------------------------------------------------- road ranges
def test_road_ranges_partition_and_balance():
    rng = np.random.default_rng(1)
    work = [int(w) for w in rng.integers(1, 10**6, 500)]
    for world in (1, 2, 3, 8):
        rs = PT.road_ranges(work, world)
        assert rs[0][0] == 0 and rs[-1][1] == len(work) and len(rs) == world
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        loads = [sum(work[a:b]) for a, b in rs]
        assert max(loads) - min(loads) <= 2 * max(work)
    rs = PT.road_ranges([5, 5], 4)                 # fewer roads than ranks: some ranges are empty
    assert len(rs) == 4 and rs[0][0] == 0 and rs[-1][1] == 2 and sum(b - a for a, b in rs) == 2
    assert PT.road_ranges([0, 0, 0, 0], 2) == [(0, 2), (2, 4)]
    assert PT.request_share(10, 3, 1) == [1, 4, 7]


SMALL_ROADS = [dict(L=int(L), N=int(N), vmax=int(v), p=float(p), seed=7, road_id=i, T=int(T))
               for i, (L, N, v, p, T) in enumerate(zip(
                   [500, 800, 1200, 300, 2000, 700, 900, 1500, 400, 1100, 650, 1800],
                   [50, 300, 100, 150, 900, 70, 450, 200, 399, 10, 325, 1000],
                   [5, 3, 8, 5, 5, 3, 8, 5, 2, 5, 3, 5],
                   [0.13, 0.0, 0.25, 0.5, 0.13, 1.0, 0.3, 0.13, 0.2, 0.13, 0.4, 0.1],
                   [40, 25, 60, 10, 35, 20, 55, 45, 30, 15, 50, 25]))]


def _road_result(r):
    x0 = O.floyd_init(r["L"], r["N"], r["seed"], r["road_id"])
    x, v, sv, cr = O.agent_run(r["L"], x0, np.zeros(r["N"], np.uint8), r["vmax"], r["p"], r["seed"], r["road_id"],
                               0, r["T"])
    return (x.tobytes(), v.tobytes(), sv.tobytes(), cr.tobytes())


def _partition_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, last = PT.rank_range(SMALL_ROADS, world, rank)
    mine = {i: _road_result(SMALL_ROADS[i]) for i in range(first, last)}
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        union = {}
        for d in gathered:
            assert not (set(d) & set(union)), "a road ran on two ranks"
            union.update(d)
        out["union"] = union
    out[f"range{rank}"] = (first, last)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_a_batch_by_road_range():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_partition_rank, args=(r, 2, port, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(180)
            assert pr.exitcode == 0
        union = dict(out["union"])
        r0, r1 = out["range0"], out["range1"]
    assert r0[0] == 0 and r0[1] == r1[0] and r1[1] == len(SMALL_ROADS) and 0 < r0[1] < len(SMALL_ROADS)
    assert sorted(union) == list(range(len(SMALL_ROADS)))
    for i, r in enumerate(SMALL_ROADS):
        assert union[i] == _road_result(r), i
