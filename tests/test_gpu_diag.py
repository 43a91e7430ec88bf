"""Diagnostics of the library: the guard band of never-written padding
columns stays zero through every kernel variant, boundary kind, batch and
reverse sweep (no stray writes; a stand-in for a memory checker), and a
bounded device wait that runs out is reported as MRT_ETIMEOUT while the
context stays usable."""
import numpy as np
import pytest

from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W

pytestmark = pytest.mark.gpu

VARIANTS = [(Bd.KERNEL_TMA, t) for t in (1, 2, 3, 4, 5, 6, 7)] + [(Bd.KERNEL_DIRECT, 0), (Bd.KERNEL_SPLIT, 0)]
BCS = [(Bd.BC_PERIODIC, Bd.BC_PERIODIC), (Bd.BC_FIXED_EQ, Bd.BC_PERIODIC),
       (Bd.BC_REFLECT_FIXED, Bd.BC_REFLECT_FIXED), (Bd.BC_FIXED_EQ, Bd.BC_FIXED_EQ)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    yield


@pytest.mark.parametrize("bcx,bcy", BCS)
def test_guard_band_after_steps(bcx, bcy):
    # 300 x 37: a ragged last strip; 1100 x 200: enough items for the queue tiles
    for nx, ny in ((300, 37), (1100, 200)):
        w = W.random_smooth(nx, ny, seed=nx, amp=0.05, bc_x=bcx, bc_y=bcy)
        for prec in (Bd.FP32, Bd.FP64):
            for kernel, tile in VARIANTS:
                with Bd.Grid.from_workload(w, precision=prec, kernel=kernel, tile=tile) as g:
                    g.step(5)
                    assert g.health() == Bd.MRT_OK
                    assert g.debug_padding() == 0, (nx, ny, prec, kernel, tile)


def test_guard_band_after_batch_and_reverse_sweep():
    ws = W.riemann_instances(count=6, seed=3, nx_range=(129, 700), ny_choices=(4, 37), nsteps=0)
    ws.append(W.random_smooth(200, 21, seed=2, amp=0.05, bc_x=Bd.BC_REFLECT_FIXED))
    with Bd.Batch(ws) as b:
        for tile, rows in ((4, 32), (5, 8), (2, 16)):
            b.tune(tile, rows)
            b.step(5)
        for i in range(len(ws)):
            assert b.grid(i).debug_padding() == 0, i
    w = W.smooth_vortex(n=256, nsteps=20, r0=0.15)
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as g:
        g.adjoint_record(w.rho, w.ux, w.uy, w.T, 20, 5)
        g.adjoint_backward(np.full((w.ny, w.nx), w.dx * w.dx))
        assert g.debug_padding() == 0


def test_bounded_wait_runs_out_and_is_reported():
    w = W.random_smooth(64, 16, seed=1, amp=0.05)
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as g:
        assert g.health() == Bd.MRT_OK
        g.debug_wait_timeout()            # about 2 s on the device
        assert g.health() == Bd.MRT_ETIMEOUT
        with pytest.raises(Bd.MrtError) as ei:
            g.totals()
        assert ei.value.code == Bd.MRT_ETIMEOUT
    # the context is still usable
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as g:
        g.step(3)
        assert g.health() == Bd.MRT_OK


def test_fma_rate_is_plausible():
    """The multiply-add throughput probe: positive, FP32 well above FP64 on
    this part, and both below the SM count times the widest issue a clock
    allows (128 FP32 lanes per SM, 2 flops each, at 3 GHz)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r64, ms64 = Bd.fma_rate(Bd.FP64, iters=200)
    r32, ms32 = Bd.fma_rate(Bd.FP32, iters=2000)
    assert 0 < r64 < r32 <= sms * 128 * 2 * 3e9
    assert ms64 > 0 and ms32 > 0
    # a warp with one active lane counts one lane's flops
    r1, _ = Bd.fma_rate(Bd.FP32, iters=200, blocks_per_sm=1, threads_per_block=32, active_lanes=1)
    assert 0 < r1 < r32
    us_stream, us_graph = Bd.launch_period(200)
    assert 0 < us_stream < 1000 and 0 < us_graph < 1000
