"""The parameter-file runner (python -m paper_2309_14311_gb300 params.ini) on
the handout's reference case: its files against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import __main__ as R

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("layout", ["agent", "grid"])
def test_reference_case_files(tmp_path, layout):
    pre = str(tmp_path / "traffic")
    text = f"L = 1000\nT = 1000\nN = 200\np = 0.13\nvmax = 5\nseed = 1\noutputprefix = {pre}\nper = 100\n"
    (tmp_path / "test.ini").write_text(text)
    assert R.main([str(tmp_path / "test.ini"), "--layout", layout, "--width", "250"]) == 0
    velo = np.load(pre + "-velo.npy")
    dens = np.load(pre + "-dens.npy")
    times = np.load(pre + "-time.npy")
    stats = np.load(pre + "-stats.npy")
    assert velo.shape == (11, 1000) and list(times) == list(range(0, 1001, 100))
    x, v = O.floyd_init(1000, 200, 1, 0), np.zeros(200, np.uint8)
    sums, crosses = [], []
    for j in range(11):
        assert np.array_equal(velo[j], O.agent_to_grid(1000, x, v)), j
        assert np.array_equal(dens[j], (velo[j] >= 0).astype(np.uint8))
        if j < 10:
            x, v, sv, cr = O.agent_run(1000, x, v, 5, 0.13, 1, 0, 100 * j, 100)
            sums.append(sv)
            crosses.append(cr)
    assert np.array_equal(stats[0], np.concatenate(sums)) and np.array_equal(stats[1], np.concatenate(crosses))
    with open(pre + "-spacetime.pgm", "rb") as f:
        assert f.read(14) == b"P5\n250 10\n255\n"
