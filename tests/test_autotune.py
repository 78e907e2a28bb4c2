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
