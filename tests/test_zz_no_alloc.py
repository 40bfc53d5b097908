"""The allocation-free alignment entry point against the oracle and the
regular entry point.

mine_align_matrix_noalloc serves callers that cannot allocate device memory
when they call in (a process whose memory manager owns the device heap, or
code that must not touch the allocator).  Its scratch is one static device
array shared by every call, so two calls in a row must each give exactly what
the CPU oracle and mine_align_matrix give on the same input; a large call
followed by a small one checks that nothing left behind in the array leaks
into the next result.  The sizes reach the array's 1024 x 1024 limit, where
the row-major copy and the direction codes fill their regions exactly.  This
file is collected last so that a run that stops at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1509_08639_gb300 import mine, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = mine.Context(device=0)
    yield c
    c.close()


def _case(rng, S, T, kind):
    if kind == 0:
        return synth.random_matrix(rng, S, T, lo=0, hi=65536), -65536, 32768
    if kind == 1:
        return synth.random_matrix(rng, S, T, values=[0, 1, 2]), -1, 0
    return (synth.random_matrix(rng, S, T, lo=-65536, hi=65536),
            -int(rng.integers(0, 70000)), int(rng.integers(-65536, 65536)))


def test_noalloc_matches_oracle_twice_in_a_row(ctx):
    rng = np.random.default_rng(2024)
    sizes = [(1024, 1024), (37, 45), (1024, 1), (1, 1), (129, 300), (0, 7), (1, 1024), (640, 512),
             (1000, 1024)]
    for S, T in sizes:
        for kind in range(3):
            M, g, th = _case(rng, S, T, kind)
            want = O.align(M, [(g, th)])[0]
            assert ctx.align_matrix(M, g, th) == want, (S, T, kind)
            first = mine.align_matrix_noalloc(M, g, th)
            second = mine.align_matrix_noalloc(M, g, th)
            assert first == want, (S, T, kind)
            assert second == want, (S, T, kind)


def test_noalloc_on_a_caller_stream():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2025)
    st = torch.cuda.Stream(device=0)
    for S, T in ((300, 700), (1024, 1024)):
        M, g, th = _case(rng, S, T, 2)
        want = O.align(M, [(g, th)])[0]
        assert mine.align_matrix_noalloc(M, g, th, stream=st) == want
        assert mine.align_matrix_noalloc(M, g, th, stream=st) == want


def test_noalloc_rejects_sizes_beyond_its_array():
    with pytest.raises(mine.MineError) as e:
        mine.align_matrix_noalloc(np.zeros((1025, 3), np.int32), -1, 0)
    assert e.value.code == -1
    with pytest.raises(mine.MineError) as e:
        mine.align_matrix_noalloc(np.zeros((3, 1025), np.int32), -1, 0)
    assert e.value.code == -1
