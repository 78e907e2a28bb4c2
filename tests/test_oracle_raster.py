"""Pins of the oracle's space-time raster row (Fig. 1): a row worked by hand,
and the special cases the definition fixes (empty road, full road, one pixel
per cell, one pixel for the whole road)."""
import numpy as np
import pytest

from oracle import oracle as O
from tests import _golden


def test_hand_worked_row():
    fx = _golden.load("raster_L10_W3.txt")
    row = O.raster_row(fx["L"], np.array(fx["x"]), fx["width"])
    assert row.tolist() == fx["row"]


@pytest.mark.parametrize("L,W", [(10, 3), (1000, 7), (4096, 4096), (12345, 100)])
def test_empty_and_full_roads(L, W):
    assert not O.raster_row(L, np.array([], dtype=np.int64), W).any()
    assert (O.raster_row(L, np.arange(L), W) == 255).all()


def test_one_pixel_per_cell_is_the_occupancy():
    rng = np.random.default_rng(5)
    L = 500
    x = np.sort(rng.choice(L, 123, replace=False))
    occ = np.zeros(L, np.uint8)
    occ[x] = 255
    assert np.array_equal(O.raster_row(L, x, L), occ)


def test_one_pixel_is_the_density():
    L, N = 1000, 237
    x = np.arange(N) * 4
    assert O.raster_row(L, x, 1).tolist() == [255 * N // L]


def test_large_road_pixel_bounds_agree_with_small_road_rule():
    # above 2^24 cells the pixels' cell counts come from ceil(i * L / W);
    # on a road just past that size they must match counting cell by cell
    L, W = (1 << 24) + 12345, 977
    counts = np.bincount((np.arange(L, dtype=np.int64) * W) // L, minlength=W)
    x = np.arange(0, L, 3)
    cars = np.bincount((x * W) // L, minlength=W)
    assert np.array_equal(O.raster_row(L, x, W), ((255 * cars) // counts).astype(np.uint8))
