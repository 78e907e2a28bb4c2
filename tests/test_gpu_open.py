"""Open roads (nasch_create_open: entry before cell 0 with probability
alpha, exit after cell L-1 open with probability beta) against the oracle's
open road, element by element: cells after T steps and the per-step sums
and exits."""
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


CASES = [  # (L, N, vmax, p, alpha, beta, T)
    (40000, 4000, 5, 0.13, 0.3, 0.7, 50),
    (2016 * 3 + 7, 1500, 5, 0.25, 0.9, 0.2, 60),   # ragged last tile
    (1000, 200, 5, 0.13, 0.5, 0.5, 100),           # the road fits one tile
    (5000, 0, 5, 0.3, 1.0, 1.0, 80),               # starts empty: the entry fills it
    (3000, 2500, 3, 0.5, 1.0, 0.0, 60),            # dense, exit closed: a jam grows back
    (20000, 3000, 20, 0.3, 0.5, 0.5, 40),          # vmax > 16: wider halos
    (12000, 3000, 5, 0.0, 0.4, 1.0, 40),           # p = 0
    (12000, 3000, 5, 1.0, 0.4, 1.0, 40),           # p = 1
    (7, 3, 2, 0.5, 0.5, 0.5, 30),                  # a tiny road
]


@pytest.mark.parametrize("L,N,vmax,p,alpha,beta,T", CASES)
def test_open_road_matches_oracle(L, N, vmax, p, alpha, beta, T):
    seed, road = 21 + L % 13, 4
    x0 = O.floyd_init(L, N, seed, road)
    c0 = O.agent_to_grid(L, x0, np.zeros(N, np.uint8))
    oc, osv, ocr = O.open_run(c0, vmax, p, alpha, beta, seed, road, 0, T)
    with NS.Road(L, N, vmax, p, seed, road, layout="grid", open=(alpha, beta)) as r:
        r.run(T)
        sv, cr = r.stats()
        assert np.array_equal(sv, osv) and np.array_equal(cr, ocr)
        assert np.array_equal(r.read_grid(), oc)


def test_resume_with_another_car_count_and_output():
    L, vmax, p, alpha, beta, seed = 30000, 5, 0.2, 0.6, 0.4, 3
    rng = np.random.default_rng(8)
    x = np.sort(rng.choice(L, 2222, replace=False)).astype(np.int32)
    v = rng.integers(0, vmax + 1, len(x)).astype(np.uint8)
    c0 = O.agent_to_grid(L, x, v)
    with NS.Road(L, 100, vmax, p, seed, 0, layout="grid", open=(alpha, beta)) as r:
        r.set_state(x, v, 500)                       # 2222 cars, not the 100 it was made with
        snaps = np.zeros((3, L), np.int8)
        r.run_output(30, 10, snaps, None)
        c = c0
        for j in range(3):
            c, _, _ = O.open_run(c, vmax, p, alpha, beta, seed, 0, 500 + 10 * j, 10)
            assert np.array_equal(snaps[j], c), j
        with pytest.raises(NS.NaschError):
            r.read_state()


def test_open_road_refusals():
    lib = NS.load()
    with pytest.raises(NS.NaschError):
        NS.Road(1000, 10, 5, 0.1, 1, layout="agent", open=(0.5, 0.5))
    for a, b in ((-0.1, 0.5), (0.5, 1.5), (float("nan"), 0.5)):
        with pytest.raises(NS.NaschError):
            NS.Road(1000, 10, 5, 0.1, 1, layout="grid", open=(a, b))
    with NS.Road(1000, 10, 5, 0.1, 1, layout="grid", open=(0.5, 0.5)) as r:
        with pytest.raises(NS.NaschError):
            r.set_state(np.arange(1001, dtype=np.int32), np.zeros(1001, np.uint8), 0)   # more cars than cells
