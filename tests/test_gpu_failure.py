"""Failure detection without a GPU fault.

A kernel's bounded wait is made to run out (an mbarrier that nothing
completes); the kernel must record the timeout in its status word and
return, the host must see NASCH_ETIMEOUT, and the context must stay usable:
a road run afterwards is still bit-exact.  Host-side faults (bad arguments,
budget overflow, cancellation) are covered by the batch and serving tests.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2309_14311_gb300 import nasch as NS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_14311_gb300 import build
    build.build()
    NS.load()


def test_bounded_wait_times_out_and_reports():
    st, word = NS.selftest_bounded_wait(50)
    assert st == NS.ETIMEOUT
    assert word & 1


def test_context_usable_after_a_timeout():
    NS.selftest_bounded_wait(20)
    L, N, T = 50000, 6000, 30
    with NS.Road(L, N, 5, 0.13, 4, layout="grid", k=4, tile=8192) as r:
        r.run(T)
        sv, _ = r.stats()
        grid = r.read_grid()
    x0 = O.floyd_init(L, N, 4, 0)
    ox, ov, osv, _ = O.agent_run(L, x0, np.zeros(N, np.uint8), 5, 0.13, 4, 0, 0, T)
    assert np.array_equal(sv, osv) and np.array_equal(grid, O.agent_to_grid(L, ox, ov))


def test_bad_arguments_are_refused():
    with pytest.raises(NS.NaschError) as e:
        NS.Road(100, 101, 5, 0.1, 1)
    assert e.value.status == NS.EINVAL
    st, _ = NS.selftest_bounded_wait(0)
    assert st == NS.EINVAL
