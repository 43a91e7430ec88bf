"""Asynchronous totals read (mrt_conserved_totals_async / mrt_totals_wait):
the pipelined use (step n+1 launched before the totals of step n are
waited for) returns, step by step, the same totals bit for bit as the
synchronous read of an identical grid; the flag word reports a tripped
timeout; tickets are checked."""
import numpy as np
import pytest

from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    return t


@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
def test_pipelined_async_totals_match_synchronous(torch, prec):
    w = W.random_smooth(300, 37, seed=5, amp=0.1)
    nsteps = 12
    with Bd.Grid.from_workload(w, precision=prec) as a:
        want = []
        for _ in range(nsteps):
            a.step(1)
            want.append(a.totals())
    stage = [torch.empty(5, dtype=torch.float64).pin_memory() for _ in range(3)]
    got = []
    with Bd.Grid.from_workload(w, precision=prec) as b:
        pending = []
        for k in range(nsteps):
            b.step(1)
            pending.append((b.totals_async(stage[k % 3]), k % 3))
            if len(pending) == 2:              # one step in flight while the previous is read
                t, slot = pending.pop(0)
                b.totals_wait(t)
                got.append(stage[slot].numpy().copy())
        for t, slot in pending:
            b.totals_wait(t)
            got.append(stage[slot].numpy().copy())
    for k in range(nsteps):
        assert got[k][4] == 0.0
        np.testing.assert_array_equal(got[k][:4], want[k])


def test_flag_word_and_tickets(torch):
    w = W.random_smooth(64, 16, seed=1, amp=0.05)
    dst = torch.full((5,), np.nan, dtype=torch.float64).pin_memory()
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as g:
        with pytest.raises(Bd.MrtError) as ei:
            g.totals_wait(0)                   # nothing issued yet
        assert ei.value.code == Bd.MRT_EINVAL
        t0 = g.totals_async(dst)               # state after creation: totals computed on request
        g.totals_wait(t0)
        np.testing.assert_array_equal(dst.numpy()[:4], g.totals())
        assert dst.numpy()[4] == 0.0
        tickets = [g.totals_async(dst) for _ in range(12)]
        g.totals_wait(tickets[0])              # its marker was reused: waits for a later copy
        g.totals_wait(tickets[-1])
        with pytest.raises(Bd.MrtError) as ei:
            g.totals_wait(tickets[-1] + 1)
        assert ei.value.code == Bd.MRT_EINVAL
        g.debug_wait_timeout()
        g.step(1)
        t = g.totals_async(dst)
        g.totals_wait(t)
        assert int(dst.numpy()[4]) & 2
