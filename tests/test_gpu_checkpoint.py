"""Checkpoint and resume through a file (mrt_save / mrt_load): a run saved
after n steps and resumed in a fresh grid, created from different fields,
continues bit for bit like the uninterrupted run (fixed-equilibrium ghosts
travel in the file), in both precisions, for periodic, fixed and walled
axes and both advection operators; the step count is restored; a grid that
does not match, a truncated file and a corrupted payload are rejected."""
import os

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


@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
@pytest.mark.parametrize("bcx,bcy,adv", [(0, 0, 0), (1, 0, 0), (2, 1, 0), (1, 1, 1), (2, 0, 1)])
def test_resume_is_bit_identical(tmp_path, prec, bcx, bcy, adv):
    w = W.random_smooth(300, 37, seed=6, amp=0.1, bc_x=bcx, bc_y=bcy)
    other = W.random_smooth(300, 37, seed=7, amp=0.1, bc_x=bcx, bc_y=bcy)   # different initial fields
    path = str(tmp_path / "state.mrt")
    with Bd.Grid.from_workload(w, precision=prec, advection=adv) as a:
        a.step(7)
        a.save(path)
        a.step(9)
        want = a.get_f()
        want_tot = a.totals()
    with Bd.Grid.from_workload(other, precision=prec, advection=adv) as b:
        b.load(path)
        assert b.info()["steps"] == 7
        b.step(9)
        np.testing.assert_array_equal(b.get_f(), want)
        np.testing.assert_array_equal(b.totals(), want_tot)
        assert b.info()["steps"] == 16


def test_mismatch_truncation_and_corruption_are_rejected(tmp_path):
    w = W.random_smooth(64, 16, seed=1, amp=0.05)
    path = str(tmp_path / "s.mrt")
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as g:
        g.step(2)
        g.save(path)
    size = os.path.getsize(path)
    cases = {
        "size": W.random_smooth(65, 16, seed=1, amp=0.05),
        "rates": W.random_smooth(64, 16, seed=1, amp=0.05, sigma=0.07),
    }
    for name, w2 in cases.items():
        with Bd.Grid.from_workload(w2, precision=Bd.FP32) as g:
            with pytest.raises(Bd.MrtError) as ei:
                g.load(path)
            assert ei.value.code == Bd.MRT_EINVAL, name
    with Bd.Grid.from_workload(w, precision=Bd.FP64) as g:
        with pytest.raises(Bd.MrtError):
            g.load(path)
    data = open(path, "rb").read()
    bad = bytearray(data)
    bad[size // 2] ^= 0x40
    for blob in (data[: size - 100], bytes(bad), b"not a checkpoint"):
        p2 = str(tmp_path / "bad.mrt")
        open(p2, "wb").write(blob)
        with Bd.Grid.from_workload(w, precision=Bd.FP32) as g:
            with pytest.raises(Bd.MrtError) as ei:
                g.load(p2)
            assert ei.value.code == Bd.MRT_EINVAL
            assert "checkpoint" in str(ei.value)
