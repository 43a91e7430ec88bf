"""GPU parity of the unsplit two-dimensional Lax-Wendroff operator
(MRT_ADV_LW2D: the axis-by-axis operator plus the mixed term on the diagonal
velocities) against the FP64 oracle's ADV_LW2D step, through the C ABI.

Tolerances as for the method's operator: FP64 1e-13 of max|f| for one raw
step and 1e-12 relative for macroscopic fields over many steps, FP32 2e-6 of
max|f| for one step from the GPU's own state and 1e-5 relative on smooth
flow.  Cases span ragged 128-column strips, every boundary combination
(the corner ghosts beyond two non-periodic ends included), the kernels that
run it (direct; TMA tiles 1, 4 and 7; the automatic choice), the queue tile
on a grid with enough work items, and the rejection of the combinations
that do not take it."""
import numpy as np
import pytest

import oracle
from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W
from _parity import assert_parity

pytestmark = pytest.mark.gpu

VARIANTS = [(Bd.KERNEL_TMA, t) for t in (0, 1, 4, 7)] + [(Bd.KERNEL_DIRECT, 0)]
BCS = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (2, 1), (0, 2), (2, 2)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    yield


def _oracle(w, nsteps):
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y,
                      advection=oracle.ADV_LW2D)
    oracle.run(g, nsteps)
    return g


def _gpu(w, prec, kernel, tile):
    return Bd.Grid.from_workload(w, precision=prec, kernel=kernel, tile=tile, advection=Bd.ADV_LW2D)


@pytest.mark.parametrize("kernel,tile", VARIANTS)
@pytest.mark.parametrize("bcx,bcy", BCS)
def test_one_step_raw_state_fp64(kernel, tile, bcx, bcy):
    w = W.random_smooth(300, 37, seed=4, amp=0.1, bc_x=bcx, bc_y=bcy)
    g = _oracle(w, 1)
    with _gpu(w, Bd.FP64, kernel, tile) as grid:
        grid.step(1)
        f = grid.get_f()
    assert np.max(np.abs(f - g.f)) <= 1e-13 * np.max(np.abs(g.f))


@pytest.mark.parametrize("kernel,tile", VARIANTS)
@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 1), (2, 0)])
def test_one_step_raw_state_fp32(kernel, tile, bcx, bcy):
    w = W.random_smooth(300, 37, seed=4, amp=0.1, bc_x=bcx, bc_y=bcy)
    with _gpu(w, Bd.FP32, kernel, tile) as grid:
        f0 = grid.get_f().astype(np.float64)
        grid.step(1)
        f1 = grid.get_f().astype(np.float64)
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y,
                      advection=oracle.ADV_LW2D)
    want = oracle.step(g, f0)
    assert np.max(np.abs(f1 - want)) <= 2e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("kernel,tile", VARIANTS)
@pytest.mark.parametrize("bcx,bcy", [(0, 0), (2, 0), (1, 1), (2, 2)])
def test_many_steps_parity(kernel, tile, bcx, bcy):
    """Ghost columns, rows and corners refreshed by the step itself (periodic
    and wall axes) stay consistent over many steps; odd count (buffers
    swapped)."""
    w = W.random_smooth(127, 130, seed=9, amp=0.1, bc_x=bcx, bc_y=bcy)
    want = oracle.macro(_oracle(w, 41))
    with _gpu(w, Bd.FP64, kernel, tile) as grid:
        grid.step(41)
        assert_parity(grid.macro(), want, linf=1e-12, label="fp64")
    with _gpu(w, Bd.FP32, kernel, tile) as grid:
        grid.step(41)
        assert_parity(grid.macro(), want, linf=1e-5, l1=1e-5, label="fp32")


def test_queue_tile_on_a_large_grid_and_totals():
    """2048 x 2048 gives every resident CTA at least two 32-row items, so the
    automatic choice is the queue tile 7 in both precisions; one FP64 step
    and its totals match the oracle."""
    w = W.random_smooth(2048, 2048, seed=3, amp=0.05)
    g = _oracle(w, 1)
    with _gpu(w, Bd.FP32, Bd.KERNEL_AUTO, 0) as grid:
        assert grid.info()["tile"] == 7
    with _gpu(w, Bd.FP64, Bd.KERNEL_AUTO, 0) as grid:
        assert grid.info()["tile"] == 7
        grid.step(1)
        f = grid.get_f()
        t = grid.totals()
    assert np.max(np.abs(f - g.f)) <= 1e-13 * np.max(np.abs(g.f))
    np.testing.assert_allclose(t, oracle.totals(g), rtol=1e-12, atol=1e-13 * np.max(np.abs(t)))


def test_four_quadrants_corners():
    """Fixed ends on both axes: the corner ghosts hold the corner cells'
    initial f (oracle reading), in both precisions and both kernels."""
    w = W.four_quadrant_riemann(n=100)
    want = oracle.macro(_oracle(w, 200))
    for kernel in (Bd.KERNEL_TMA, Bd.KERNEL_DIRECT):
        with _gpu(w, Bd.FP64, kernel, 0) as grid:
            grid.step(200)
            assert_parity(grid.macro(), want, linf=1e-11, label="fp64")
        with _gpu(w, Bd.FP32, kernel, 0) as grid:
            grid.step(200)
            assert_parity(grid.macro(), want, l1=1e-4, label="fp32")


@pytest.mark.parametrize("kernel,tile", [(Bd.KERNEL_TMA, 1), (Bd.KERNEL_TMA, 4), (Bd.KERNEL_TMA, 7),
                                         (Bd.KERNEL_DIRECT, 0)])
def test_guard_band_and_minimum_grid(kernel, tile):
    """No write lands outside the ghost ring (the corner stores included), and
    the 3 x 3 minimum grid, whose corner cells feed every ghost, matches."""
    for bcx, bcy in BCS:
        w = W.random_smooth(3, 3, seed=2, amp=0.05, bc_x=bcx, bc_y=bcy)
        g = _oracle(w, 5)
        with _gpu(w, Bd.FP64, kernel, tile) as grid:
            grid.step(5)
            assert np.max(np.abs(grid.get_f() - g.f)) <= 1e-13 * np.max(np.abs(g.f)), (bcx, bcy)
            assert grid.debug_padding() == 0
        w = W.random_smooth(300, 37, seed=2, amp=0.05, bc_x=bcx, bc_y=bcy)
        for prec in (Bd.FP32, Bd.FP64):
            with _gpu(w, prec, kernel, tile) as grid:
                grid.step(4)
                assert grid.health() == Bd.MRT_OK
                assert grid.debug_padding() == 0, (bcx, bcy, prec)


def test_rejected_combinations():
    w = W.random_smooth(64, 16, seed=1, amp=0.05)
    for tile in (2, 3, 5, 6):
        with pytest.raises(Bd.MrtError) as ei:
            _gpu(w, Bd.FP32, Bd.KERNEL_TMA, tile)
        assert ei.value.code == Bd.MRT_EINVAL
    with pytest.raises(Bd.MrtError) as ei:
        Bd.Grid.from_workload(w, precision=Bd.FP32, advection=2)
    assert ei.value.code == Bd.MRT_EINVAL
    with _gpu(w, Bd.FP32, Bd.KERNEL_AUTO, 0) as grid:
        with pytest.raises(Bd.MrtError) as ei:
            grid.adjoint_record(w.rho, w.ux, w.uy, w.T, 4, 2)
        assert ei.value.code == Bd.MRT_EINVAL
