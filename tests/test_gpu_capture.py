"""mrt_step inside a caller's CUDA graph capture of the grid's stream.

Inside a capture the library launches every step directly and reduces the
totals on the grid's stream into a totals slot of the graph's own (its own
two-step graphs and the side-stream reduction stay out of the caller's
graph).  Replays of an even step count on the grid's stream advance the state
bit for bit as direct calls do; replays and direct calls of even step counts
may alternate, and the totals read afterwards are those of the latest step,
whichever of the two produced it (a stamp of the stream order decides).
"""
import numpy as np
import pytest

from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    yield


def _steps(g, n, kernel):
    """n steps on a reference grid with the kernel a capture launches: the
    split kernel's multi-step launch is not taken inside a capture, so its
    reference steps one at a time (the same kernel, bit for bit)."""
    if kernel == Bd.KERNEL_SPLIT:
        for _ in range(n):
            g.step(1)
    else:
        g.step(n)


@pytest.mark.parametrize("kernel,tile", [(Bd.KERNEL_TMA, 6), (Bd.KERNEL_TMA, 4), (Bd.KERNEL_DIRECT, 0),
                                         (Bd.KERNEL_SPLIT, 0)])
@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
def test_captured_steps_replay_like_direct_calls(kernel, tile, prec):
    import torch
    w = W.random_smooth(700, 150, seed=13, amp=0.1, bc_x=Bd.BC_FIXED_EQ)
    s = torch.cuda.Stream()
    with Bd.Grid.from_workload(w, precision=prec, kernel=kernel, tile=tile, stream=s.cuda_stream) as a, \
            Bd.Grid.from_workload(w, precision=prec, kernel=kernel, tile=tile) as b:
        # two calls: both partials buffers have a side-stream reduction
        # recorded before the capture starts
        for g in (a, b):
            _steps(g, 3, kernel)
            g.step(1)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=s):
            a.step(4)
            with pytest.raises(Bd.MrtError):
                a.totals()
        assert a.info()["steps"] == 8
        with torch.cuda.stream(s):
            for _ in range(3):
                cg.replay()
                _steps(b, 4, kernel)
                np.testing.assert_array_equal(a.get_f(), b.get_f())
                np.testing.assert_array_equal(a.totals(), b.totals())
            # direct calls on the same grid after the replays go on from the
            # replayed state
            _steps(a, 5, kernel)
            _steps(b, 5, kernel)
            np.testing.assert_array_equal(a.get_f(), b.get_f())
            np.testing.assert_array_equal(a.totals(), b.totals())
        assert a.health() == Bd.MRT_OK and b.health() == Bd.MRT_OK
        assert a.info()["steps"] == 13 and b.info()["steps"] == 21


@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
def test_direct_steps_between_capture_and_replay(prec):
    """Capture, then a direct even step, then replays and direct steps in
    turn: the state and both totals readers follow the latest step (the
    replay's totals are not hidden by the earlier direct step's, nor the
    other way round)."""
    import torch
    w = W.random_smooth(300, 70, seed=17, amp=0.1)
    s = torch.cuda.Stream()
    stage = torch.empty(5, dtype=torch.float64).pin_memory()
    with Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_TMA, tile=6, stream=s.cuda_stream) as a, \
            Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_TMA, tile=6) as b:
        a.step(2)
        b.step(2)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=s):
            a.step(2)
        with torch.cuda.stream(s):
            a.step(2)                 # direct, after the capture
            b.step(2)
            np.testing.assert_array_equal(a.totals(), b.totals())
            for direct_after in (False, True, True, False):
                cg.replay()
                b.step(2)
                if direct_after:
                    a.step(4)
                    b.step(4)
                np.testing.assert_array_equal(a.get_f(), b.get_f())
                want = b.totals()
                np.testing.assert_array_equal(a.totals(), want)
                t = a.totals_async(stage)
                cg.replay()           # enqueued while the copy may still be pending
                b.step(2)
                a.totals_wait(t)
                np.testing.assert_array_equal(stage.numpy()[:4], want)
                assert stage.numpy()[4] == 0.0
                np.testing.assert_array_equal(a.totals(), b.totals())
        assert a.health() == Bd.MRT_OK
