"""The benchmark's N > 1 path on CPU ranks (gloo, world size 2).

The large road does not shard without a halo exchange, so N GPUs run N
independent replica roads, one per rank, told apart by the Philox road id;
the whole-job rate is all ranks' vehicle-updates over the slowest rank's
time.  Here two gloo ranks run their replicas with the oracle and reduce
through the same helpers the benchmark uses."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import time

    import torch.distributed as dist

    from oracle import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    road = bench.replica_road_ids(world)[rank]
    L, N, T = 5000, 400, 50
    x0 = O.floyd_init(L, N, 1, road)
    t0 = time.perf_counter()
    x, v, sv, cr = O.agent_run(L, x0, np.zeros(N, np.uint8), 5, 0.13, 1, road, 0, T)
    secs = time.perf_counter() - t0 + 0.01 * rank
    t_max = bench.reduce_over_ranks(secs, "max", device="cpu")
    units = bench.reduce_over_ranks(float(N * T), "sum", device="cpu")
    out[rank] = (road, t_max, units, int(sv.sum()), x.tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_run_independent_replicas():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    (r0, t0, u0, s0, x0), (r1, t1, u1, s1, x1) = res[0], res[1]
    assert (r0, r1) == (0, 1)
    assert t0 == t1 and u0 == u1 == 2 * 400 * 50       # every rank sees the max time and the sum
    assert x0 != x1                                     # distinct road ids: independent replicas
    rate, t = bench.aggregate([400 * 50, 400 * 50], [t0, t1])
    assert t == t0 and rate == pytest.approx(u0 / t0)
