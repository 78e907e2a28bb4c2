"""GPU parity of the domain-decomposed road (nasch_segment_run) against the
oracle.

The ring is split into 1, 2, 3 or 5 contiguous cell ranges, every range
held in its own device buffer with halos; the halos are exchanged between
the buffers before every launch (the exchange a multi-GPU run does by
point-to-point messages, here copies on one GPU, one rank after another, so
no kernel waits on another), and each rank's k steps run in the library's
segment kernel.  The owned cells put together, and the per-step statistics
summed over ranks, must equal the oracle's run of the whole ring, bit for
bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import decomp as DC
from paper_2309_14311_gb300 import nasch as NS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_14311_gb300 import build
    build.build()
    NS.load()
    return torch


CASES = [
    # L, N, vmax, p, k, world, T
    (200_000, 12_500, 5, 0.13, 8, 3, 67),     # many tiles per rank, ragged last launch
    (200_000, 12_500, 5, 0.13, 8, 1, 40),     # one rank: halos from itself across the ring's end
    (50_003, 20_000, 5, 0.5, 4, 2, 33),       # dense, odd length
    (60_000, 7_000, 8, 0.25, 16, 5, 48),      # vmax 8, halo 128
    (30_000, 3_000, 5, 0.0, 6, 3, 30),        # p = 0
    (30_000, 20_000, 3, 1.0, 5, 2, 17),       # p = 1
    (2**31, 40_000, 5, 0.13, 4, 2, 12),       # the largest ring: cells near 2^31 wrap
    (5_000, 1_000, 20, 0.2, 25, 2, 50),       # halo 512, the largest
]


def _run(torch, L, N, vmax, p, k, world, T, seed=4, road=9):
    x0 = O.floyd_init(L, N, seed, road)
    segs = DC.segments(L, world, k, vmax)
    bufs = []
    for s in segs:   # owned cells from the cars; the first exchange fills the halos
        b = torch.full((s.W,), -7, dtype=torch.int8)
        b[s.owned_part()] = -1
        j = (x0.astype(np.int64) - s.a) % L
        b[torch.from_numpy(s.H + j[j < s.owned])] = 0
        bufs.append(b.cuda())
    bufs, stats = DC.run_local(segs, bufs, T, DC.library_step(L, vmax, p, seed, road))
    torch.cuda.synchronize()
    owned = [b[s.owned_part()].cpu().numpy() for s, b in zip(segs, bufs)]
    sv = sum(torch.cat([st[0] for st in stats[r]]).cpu().numpy().astype(np.uint64) for r in range(world))
    cr = sum(torch.cat([st[1] for st in stats[r]]).cpu().numpy().astype(np.uint64) for r in range(world))
    ox, ov, osv, ocr = O.agent_run(L, x0, np.zeros(N, np.uint8), vmax, p, seed, road, 0, T, openmp=True)
    return segs, owned, sv, cr, ox, ov, osv, ocr


@pytest.mark.parametrize("L,N,vmax,p,k,world,T", CASES)
def test_decomposed_road_matches_oracle(torch_cuda, L, N, vmax, p, k, world, T):
    segs, owned, sv, cr, ox, ov, osv, ocr = _run(torch_cuda, L, N, vmax, p, k, world, T)
    assert np.array_equal(sv, osv) and np.array_equal(cr, ocr), "statistics summed over ranks"
    if L <= 1 << 24:
        assert np.array_equal(np.concatenate(owned), O.agent_to_grid(L, ox, ov))
    else:   # compare the cars each rank owns
        got_x = np.concatenate([s.a + np.flatnonzero(o >= 0) for s, o in zip(segs, owned)])
        got_v = np.concatenate([o[o >= 0] for o in owned]).astype(np.uint8)
        order = np.argsort(ox, kind="stable")
        assert np.array_equal(got_x, ox[order].astype(np.int64)) and np.array_equal(got_v, ov[order])


def test_segment_run_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    a = torch.full((1024 + 64,), -1, dtype=torch.int8, device="cuda")
    b = torch.full((1024 + 64,), -1, dtype=torch.int8, device="cuda")
    sv = torch.zeros(8, dtype=torch.int64, device="cuda")
    cr = torch.zeros(8, dtype=torch.int64, device="cuda")
    ok = dict(owned=1024, halo=32, first_cell=0, L=4096, vmax=5, p=0.1, seed=1, road_id=0, step0=0, k=4)

    def call(src=a, dst=b, **kw):
        args = dict(ok, **kw)
        NS.segment_run(src.data_ptr(), dst.data_ptr(), args["owned"], args["halo"], args["first_cell"], args["L"],
                       args["vmax"], args["p"], args["seed"], args["road_id"], args["step0"], args["k"],
                       sv.data_ptr(), cr.data_ptr())

    call()
    torch.cuda.synchronize()
    for bad in (dict(halo=24), dict(halo=16), dict(halo=528, k=64), dict(k=0), dict(first_cell=4096),
                dict(owned=0), dict(p=1.5), dict(vmax=128)):
        with pytest.raises(NS.NaschError) as e:
            call(**bad)
        assert e.value.status == NS.EINVAL, bad
    with pytest.raises(NS.NaschError):
        call(dst=a)                                    # in place
    with pytest.raises(NS.NaschError):
        call(src=a[1:])                                # not 16-byte aligned
