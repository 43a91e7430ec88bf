"""GPU parity of the unsplit two-dimensional Lax-Wendroff operator
(MRT_ADV_LW2D: the axis-by-axis operator plus the mixed term on the diagonal
velocities) against the FP64 oracle's ADV_LW2D step, through the C ABI.

Tolerances as for the method's operator: FP64 1e-13 of max|f| for one raw
step and 1e-12 relative for macroscopic fields over many steps, FP32 2e-6 of
max|f| for one step from the GPU's own state and 1e-5 relative on smooth
flow.  Cases span ragged 128-column strips, every boundary combination
(the corner ghosts beyond two non-periodic ends included), the kernels that
run it (direct; TMA tiles 1, 4, 5, 6 and 7; the automatic choice), the queue tile
on a grid with enough work items, the rejection of the combinations that
do not take it, and the reverse mode (one reverse step and whole-run
gradients against the oracle's reverse mode of the same operator)."""
import numpy as np
import pytest

import oracle
from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W
from _parity import assert_parity

pytestmark = pytest.mark.gpu

VARIANTS = [(Bd.KERNEL_TMA, t) for t in (0, 1, 4, 5, 6, 7)] + [(Bd.KERNEL_DIRECT, 0), (Bd.KERNEL_SPLIT, 0)]
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
    """2048 x 2048 gives every resident CTA at least two work items (10 rows
    each for this operator, the last band ragged), so the automatic choice
    is the queue tile 6 in both precisions; one FP64 step and its totals
    match the oracle."""
    w = W.random_smooth(2048, 2048, seed=3, amp=0.05)
    g = _oracle(w, 1)
    with _gpu(w, Bd.FP32, Bd.KERNEL_AUTO, 0) as grid:
        assert grid.info()["tile"] == 6
    with _gpu(w, Bd.FP64, Bd.KERNEL_AUTO, 0) as grid:
        assert grid.info()["tile"] == 6
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


@pytest.mark.parametrize("kernel,tile", [(Bd.KERNEL_TMA, t) for t in (1, 4, 5, 6, 7)] + [(Bd.KERNEL_DIRECT, 0)])
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
    for tile in (2, 3):
        with pytest.raises(Bd.MrtError) as ei:
            _gpu(w, Bd.FP32, Bd.KERNEL_TMA, tile)
        assert ei.value.code == Bd.MRT_EINVAL
    with pytest.raises(Bd.MrtError) as ei:
        Bd.Grid.from_workload(w, precision=Bd.FP32, advection=2)
    assert ei.value.code == Bd.MRT_EINVAL
    # batches take the axis-by-axis operator only
    import ctypes
    L = Bd.load()
    p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, w.s, w.bc_x, w.bc_y, Bd.FP32, advection=Bd.ADV_LW2D)
    params = (Bd.Params * 1)(p)
    arrs = [np.ascontiguousarray(np.broadcast_to(a, (w.ny, w.nx)), dtype=np.float64)
            for a in (w.rho, w.ux, w.uy, w.T)]
    ptrs = [(ctypes.c_void_p * 1)(a.ctypes.data) for a in arrs]
    h = ctypes.c_void_p()
    rc = L.mrt_batch_create(1, params, *(ctypes.cast(q, ctypes.POINTER(ctypes.c_void_p)) for q in ptrs), 0,
                            ctypes.byref(h))
    assert rc == Bd.MRT_EINVAL


# --------------------------------------------------------------------------
# Reverse mode of the unsplit operator
# --------------------------------------------------------------------------
def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("prec,tol", [(Bd.FP64, 1e-12), (Bd.FP32, 2e-5)])
@pytest.mark.parametrize("bcx,bcy", BCS)
def test_adjoint_step_matches_oracle(prec, tol, bcx, bcy):
    """One reverse step (direct kernel, mrt_adjoint_step) against the
    oracle's transpose of the ADV_LW2D step: lam and the rate gradients."""
    w = W.random_smooth(140, 21, seed=8, amp=0.1, bc_x=bcx, bc_y=bcy)
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y,
                      advection=oracle.ADV_LW2D)
    f = oracle.step(g)
    rng = np.random.default_rng(3)
    lam_next = rng.standard_normal(f.shape)
    dt = np.float64 if prec == Bd.FP64 else np.float32
    f_in, l_in = f.astype(dt), lam_next.astype(dt)
    gs = np.zeros(16)
    want = oracle.step_adjoint(g, f_in.astype(np.float64), l_in.astype(np.float64), np.zeros_like(g.gx),
                               np.zeros_like(g.gy), gs)
    with _gpu(w, prec, Bd.KERNEL_AUTO, 0) as grid:
        got, gs_gpu = grid.adjoint_step(f_in, l_in)
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    np.testing.assert_allclose(gs_gpu[4:], gs[4:], rtol=tol * 50, atol=tol * np.max(np.abs(gs)))


def _loss(target, dx):
    def lg(r):
        d = r - target
        return 0.5 * np.sum(d * d) * dx * dx, d * dx * dx
    return lg


@pytest.mark.parametrize("case", ["vortex", "tube", "quadrants", "walls", "wall_fixed"])
def test_adjoint_run_matches_oracle(case):
    """Gradients of L(rho_N) with respect to the initial fields and the
    rates through 30 ADV_LW2D steps (checkpoints every 7), both kernels, both
    precisions; the fixed-ghost adjoints (corners included) enter the
    gradients of the boundary cells."""
    if case == "vortex":
        w = W.smooth_vortex(n=40, nsteps=30, r0=0.15)
        target = W.vortex_target(w)
    elif case == "tube":
        w = W.sod_tube(nx=150, ny=5, nsteps=30)
        target = w.rho * 0.97 + 0.01
    elif case == "quadrants":
        w = W.shrink(W.four_quadrant_riemann(n=48), 30)
        target = w.rho * 0.97 + 0.01
    elif case == "walls":
        w = W.random_smooth(150, 37, seed=31, amp=0.1, bc_x=Bd.BC_REFLECT_FIXED, bc_y=Bd.BC_REFLECT_FIXED,
                            nsteps=30)
        target = w.rho * 0.98 + 0.02
    else:
        w = W.random_smooth(61, 37, seed=32, amp=0.1, bc_x=Bd.BC_FIXED_EQ, bc_y=Bd.BC_REFLECT_FIXED, nsteps=30)
        target = w.rho * 0.98 + 0.02
    lg = _loss(target, w.dx)
    ref = oracle.adjoint_run(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.nsteps, lg,
                             w.bc_x, w.bc_y, ckpt=7, advection=oracle.ADV_LW2D)
    for prec, tol in ((Bd.FP64, 1e-10), (Bd.FP32, 1e-3)):
        for kernel in (Bd.KERNEL_TMA, Bd.KERNEL_DIRECT):
            with _gpu(w, prec, kernel, 0) as grid:
                grid.adjoint_record(w.rho, w.ux, w.uy, w.T, w.nsteps, 7)
                L, dL = lg(grid.macro()[0])
                got = grid.adjoint_backward(dL)
            # L is half the squared misfit of two close fields: its error is
            # bounded through the field tolerance (1e-12 FP64, 1e-5 FP32 of
            # max|rho|) times sum |dL/drho|
            rho_tol = 1e-12 if prec == Bd.FP64 else 1e-5
            assert abs(L - ref[0]) <= rho_tol * np.max(np.abs(w.rho)) * 2 * np.sum(np.abs(dL)) + 1e-14 * abs(ref[0])
            for name, a, b in zip(("rho", "ux", "uy", "T"), got[:4], ref[1:5]):
                scale = max(np.linalg.norm(b), 1e-4 * max(np.linalg.norm(x) for x in ref[1:5]))
                err = np.linalg.norm(a - b) / scale
                assert err <= tol, (case, prec, kernel, name, err)
            err = np.linalg.norm(got[4] - ref[5]) / np.linalg.norm(ref[5])
            assert err <= tol, (case, prec, kernel, "rates", err)


def test_full_size_kh_sampled_windows():
    """The bench's unsplit-operator leg: 4096^2 Kelvin-Helmholtz in FP32 on
    the automatic choice (tile 6).  After 3 steps, 12 seeded 48^2 windows
    (the periodic corners, whose cells read the diagonally wrapped corner
    ghosts, and strip/item seams among them) of step 3 -> 4 match one
    ADV_LW2D oracle step on the window (exact in its interior, the stencil
    reaching one cell, diagonals included)."""
    w = W.kelvin_helmholtz(n=4096, nsteps=0)
    rng = np.random.default_rng(1)
    n = 48
    corners = [(0, 0), (w.ny - n, w.nx - n), (0, w.nx - n), (w.ny - n, 0), (2000, 128 * 16 - 24)]
    wins = corners + [(int(rng.integers(0, w.ny - n)), int(rng.integers(0, w.nx - n))) for _ in range(7)]
    with _gpu(w, Bd.FP32, Bd.KERNEL_TMA, 0) as grid:
        assert grid.info()["tile"] == 6
        grid.step(3)
        f3 = grid.get_f()
        grid.step(1)
        f4 = grid.get_f()
    for (y0, x0) in wins:
        ys = np.arange(y0 - 1, y0 + n + 1) % w.ny
        xs = np.arange(x0 - 1, x0 + n + 1) % w.nx
        fw = np.ascontiguousarray(f3[:, ys][:, :, xs].astype(np.float64))
        g = oracle.Grid(n + 2, n + 2, w.dx, w.dt, w.b, w.s, oracle.BC_PERIODIC, oracle.BC_PERIODIC,
                        oracle.ADV_LW2D)
        g.gx = np.zeros((16, 2, n + 2))
        g.gy = np.zeros((16, 2, n + 2))
        want = oracle.step(g, fw)[:, 1:-1, 1:-1]
        got = f4[:, y0:y0 + n, x0:x0 + n].astype(np.float64)
        assert np.max(np.abs(got - want)) <= 2e-6 * np.max(np.abs(want)), (y0, x0)


def test_autograd_function_with_the_unsplit_operator():
    """torch.autograd through mrt_run(advection=ADV_LW2D) in FP64 gives the
    oracle's ADV_LW2D gradients, and a central difference of the GPU loss in
    one rate (s_6, relative step 1e-4) agrees with the rate gradient."""
    import torch

    from paper_1004_5442_gb300.autograd import mrt_run
    w = W.smooth_vortex(n=40, nsteps=20, r0=0.15)
    tgt = W.vortex_target(w)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda", requires_grad=True)
    rho0, ux0, uy0, T0 = dev(w.rho), dev(w.ux), dev(w.uy), dev(w.T)
    s = torch.tensor(w.s, device="cuda", requires_grad=True)
    params = dict(nx=w.nx, ny=w.ny, dx=w.dx, dt=w.dt, gamma=w.gamma, precision=Bd.FP64,
                  advection=Bd.ADV_LW2D)
    target = torch.tensor(tgt, device="cuda")
    rhoN = mrt_run(rho0, ux0, uy0, T0, s, params, w.nsteps, 6)
    L = 0.5 * torch.sum((rhoN - target) ** 2) * w.dx ** 2
    L.backward()
    lg = _loss(tgt, w.dx)
    ref = oracle.adjoint_run(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.nsteps, lg,
                             ckpt=6, advection=oracle.ADV_LW2D)
    for t, r in zip((rho0, ux0, uy0, T0), ref[1:5]):
        assert _rel(t.grad.cpu().numpy(), r) <= 1e-10
    assert _rel(s.grad.cpu().numpy(), ref[5]) <= 1e-10

    def loss_of(sv):
        with torch.no_grad():
            r = mrt_run(rho0, ux0, uy0, T0, torch.tensor(sv, device="cuda"), params, w.nsteps, 6)
            return float(0.5 * torch.sum((r - target) ** 2) * w.dx ** 2)
    k, h = 5, 1e-4
    sp, sm = np.array(w.s), np.array(w.s)
    sp[k] *= 1 + h
    sm[k] *= 1 - h
    fd = (loss_of(sp) - loss_of(sm)) / (2 * h * w.s[k])
    got = float(s.grad[k])
    scale = float(torch.max(torch.abs(s.grad * s.detach())))
    assert abs(got - fd) * w.s[k] <= 1e-4 * abs(fd) * w.s[k] + 1e-6 * scale, (got, fd)
