"""The allocation-free entry point nasch_floyd_init_device_noalloc.

It serves callers that cannot allocate device memory (their device memory is
owned by another allocator, or allocation is forbidden after start-up): the
caller passes the output buffer and the library's scratch is a fixed device
array.  Its result must equal the existing entry point nasch_floyd_init
(exact: the output is integer cell indices), on two calls in a row - the
second call reuses the scratch left by the first - and a road longer than
the fixed scratch must be refused.  This file is collected last so that a
run stopping at the first failure has run every other test first; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest

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


def _noalloc(torch, L, N, seed, road, stream):
    out = torch.full((max(N, 1),), -7, dtype=torch.int32, device="cuda")   # the caller allocates the output
    NS.floyd_init_device_noalloc(L, N, seed, road, out.data_ptr(), stream)
    stream.synchronize()
    return out[:N].cpu().numpy()


def test_two_calls_in_a_row_match_nasch_floyd_init(torch_cuda):
    torch = torch_cuda
    stream = torch.cuda.Stream()
    cases = [(1_000_000, 300_000, 7, 3), (2**24, 2**20, 11, 0)]   # the second call reuses the first's scratch
    for L, N, seed, road in cases:
        got = _noalloc(torch, L, N, seed, road, stream)
        want = NS.floyd_init(L, N, seed, road)
        assert np.array_equal(got, want), (L, N)
    # and once more with a shorter road after a longer one (stale bits beyond L)
    got = _noalloc(torch, 5000, 1000, 5, 9, stream)
    assert np.array_equal(got, NS.floyd_init(5000, 1000, 5, 9))


def test_road_longer_than_the_scratch_is_refused(torch_cuda):
    torch = torch_cuda
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(NS.NaschError) as e:
        NS.floyd_init_device_noalloc(2**24 + 1, 4, 1, 0, out.data_ptr(), None)
    assert e.value.status == NS.EINVAL
    assert "scratch" in str(e.value)
