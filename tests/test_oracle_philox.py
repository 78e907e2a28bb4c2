"""Pins for the oracle's Philox4x32-10, slowdown threshold and draw keying.

Philox is pinned to two implementations that are not ours (cuRAND's host
generator and Triton's interpreted Philox), the threshold to exact rational
arithmetic, and the keying of the rule-3 draw (Handout, model section: slow
down iff r < p) to draws taken from those independent generators.
"""
import fractions
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import _independent_philox as IP

SEEDS = [0, 1, 1234, 0xDEADBEEF12345678, (1 << 64) - 1, 0x0000000100000000]


@pytest.mark.parametrize("seed", SEEDS)
def test_philox_matches_curand_host_generator(seed):
    n = 3 * 65536 + 17          # three counter-word-0 values, all 65536 word-2 values
    blocks = IP.curand_host_blocks(seed, n)
    if blocks is None:
        pytest.skip("cuRAND host library not available")
    ctr = IP.curand_block_counters(n)
    ours = O.philox_many(ctr, seed)
    assert np.array_equal(ours, blocks)


def test_philox_matches_triton_on_all_counter_words():
    rng = np.random.default_rng(2309)
    reqs = []
    for seed in SEEDS + [int(s) for s in rng.integers(0, 2**63, 4)]:
        ctr = rng.integers(0, 2**32, size=(256, 4), dtype=np.uint64).astype(np.uint32)
        ctr[0] = 0
        ctr[1] = [0xFFFFFFFF] * 4
        reqs.append((seed, ctr))
    res = IP.triton_philox(reqs)
    if res is None:
        pytest.skip("triton not importable")
    for (seed, ctr), theirs in zip(reqs, res):
        assert np.array_equal(O.philox_many(ctr, seed), theirs), hex(seed)


def _exact_slowdown(u, p):
    """r = u * 2^-32 < p, in exact rationals (the handout's acceptance test)."""
    return fractions.Fraction(u, 1 << 32) < fractions.Fraction(p)


@pytest.mark.parametrize("p", [0.0, 1.0, 0.5, 0.13, 0.2, 0.25, 2.0**-32, 2.0**-33, 3 * 2.0**-33,
                               math.nextafter(0.0, 1.0), math.nextafter(1.0, 0.0), 1 / 3, 0.999999])
def test_threshold_is_exact_acceptance_boundary(p):
    thr = O.slow_threshold(p)
    assert 0 <= thr <= 1 << 32
    for u in (thr - 2, thr - 1, thr, thr + 1):
        if 0 <= u < 1 << 32:
            assert (u < thr) == _exact_slowdown(u, p), (p, u, thr)


def test_threshold_random_p():
    rng = np.random.default_rng(7)
    for p in rng.random(2000):
        thr = O.slow_threshold(float(p))
        for u in (thr - 1, thr):
            if 0 <= u < 1 << 32:
                assert (u < thr) == _exact_slowdown(u, float(p))


def test_threshold_special_values():
    assert O.slow_threshold(0.0) == 0
    assert O.slow_threshold(1.0) == 1 << 32
    assert O.slow_threshold(0.5) == 1 << 31
    assert O.slow_threshold(0.13) == 558345749   # ceil(0.13 * 2^32), 0.13*2^32 = 558345748.48


def _single_car_after_one_step(cell, road, step, thr, L=1000, vmax=5):
    x, v, sv, cr = O.agent_run(L, [cell], [0], vmax, 0.0, seed=SEED_KEY, road=road, step0=step,
                               T=1, thr=thr)
    return int(v[0])


SEED_KEY = 0x0123456789ABCDEF


def test_slowdown_draw_keying_against_curand():
    """A car alone on the ring has v = 1 after rules 1-2 (from v = 0).  With the
    draw u of counter (cell, step=0, road, tag 0) taken from cuRAND, it must
    slow down under threshold u+1 and not under threshold u."""
    cases = [(0, 0), (3, 0), (7, 11), (2, 65535), (5, 1234)]
    n = max(c * 65536 + r for c, r in cases) + 1
    blocks = IP.curand_host_blocks(SEED_KEY, n)
    if blocks is None:
        pytest.skip("cuRAND host library not available")
    for cell, road in cases:
        u = int(blocks[cell * 65536 + road, 0])
        assert _single_car_after_one_step(cell, road, 0, thr=u) == 1
        assert _single_car_after_one_step(cell, road, 0, thr=u + 1) == 0


def test_slowdown_and_init_keying_against_triton():
    """Same check at step > 0 (counter word 1) with Triton's Philox, and the
    Floyd initialisation's first pick (tag 1 in counter word 3)."""
    cases = [(17, 9, 3), (999, 123456, 0), (0, 0xFFFFFFFF, 77)]  # (cell, step, road)
    ctr = np.zeros((4, 4), dtype=np.uint32)
    for i, (cell, step, road) in enumerate(cases):
        ctr[i] = [cell, step, road, 0]
    ctr[3] = [0, 0, 5, 1]   # Floyd draw m=0 for road 5
    res = IP.triton_philox([(SEED_KEY, ctr)])
    if res is None:
        pytest.skip("triton not importable")
    words = res[0]
    for i, (cell, step, road) in enumerate(cases):
        u = int(words[i, 0])
        assert _single_car_after_one_step(cell, road, step, thr=u) == 1
        assert _single_car_after_one_step(cell, road, step, thr=u + 1) == 0
    # Floyd with N = 1: the single pick is t = floor(r * L / 2^64), r = w1:w0.
    r = (int(words[3, 1]) << 32) | int(words[3, 0])
    for L in (1, 2, 1000, 2**31):
        assert O.floyd_init(L, 1, SEED_KEY, road=5)[0] == (r * L) >> 64
