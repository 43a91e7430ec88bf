"""GPU parity: the CUDA step (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances:
  FP64 GPU vs oracle      1e-12 relative (long shock runs 1e-10): only the
                          summation order differs (symmetry-adapted blocks on
                          the GPU, dense 16x16 loops in the oracle).
  FP32 GPU, smooth flow   L-inf and L1 <= 1e-5 relative per field.
  FP32 GPU, shocks        L1 <= 1e-4 relative per field.
Velocity errors are relative to the flow-speed scale of the oracle solution.
"""
import numpy as np
import pytest

import oracle
from oracle import riemann
from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W
from _parity import assert_parity, field_errors, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

KERNELS = [Bd.KERNEL_TMA, Bd.KERNEL_DIRECT]
# (kernel, tile): every compiled TMA variant, the direct and the split kernel
VARIANTS = [(Bd.KERNEL_TMA, t) for t in (1, 2, 3, 4, 5, 6, 7)] + [(Bd.KERNEL_DIRECT, 0), (Bd.KERNEL_SPLIT, 0)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    yield


# --------------------------------------------------------------------------
# Raw state after one step
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel,tile", VARIANTS)
@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_one_step_raw_state_fp64(kernel, tile, bcx, bcy):
    w = W.random_smooth(300, 37, seed=4, amp=0.1, bc_x=bcx, bc_y=bcy)
    g = run_oracle(w, 1)
    with run_gpu(w, Bd.FP64, kernel, nsteps=1, tile=tile) as grid:
        f = grid.get_f()
    scale = np.max(np.abs(g.f))
    assert np.max(np.abs(f - g.f)) <= 1e-13 * scale


@pytest.mark.parametrize("kernel,tile", VARIANTS)
@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 1)])
def test_one_step_raw_state_fp32(kernel, tile, bcx, bcy):
    w = W.random_smooth(300, 37, seed=4, amp=0.1, bc_x=bcx, bc_y=bcy)
    with Bd.Grid.from_workload(w, precision=Bd.FP32, kernel=kernel, tile=tile) as grid:
        f0 = grid.get_f().astype(np.float64)
        grid.step(1)
        f1 = grid.get_f().astype(np.float64)
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    want = oracle.step(g, f0)  # oracle step from the GPU's FP32 state
    scale = np.max(np.abs(want))
    assert np.max(np.abs(f1 - want)) <= 2e-6 * scale


@pytest.mark.parametrize("case", ["kh", "tube", "hot"])
def test_fp32_readout_of_the_fp32_state(case):
    """An FP32 grid reads rho, u, T out in double-float arithmetic (about 44
    bits per operation): against the oracle's FP64 readout of the same FP32
    state within 1e-11 of each field's scale (the closure's cancellation
    e - j^2/rho costs at most a factor of ten on these states).  Device and
    host readouts, several chunks of the latter."""
    import torch
    w = {"kh": W.kelvin_helmholtz(n=2048, nsteps=0),
         "tube": W.riemann_instances(count=1, seed=4, nx_range=(2000, 2000), ny_choices=(256,), nsteps=0)[0],
         "hot": W.random_smooth(700, 300, seed=9, amp=0.3, nsteps=0)}[case]
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as grid:
        grid.step(40)
        f = grid.get_f().astype(np.float64)
        got = grid.macro()
        dev = [torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
        grid.macro(dev)
        torch.cuda.synchronize()
    for a, b in zip(got, dev):
        np.testing.assert_array_equal(a, b.cpu().numpy())
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    want = oracle.macro(g, f)
    errs = assert_parity(got, want, linf=1e-11, label=f"readout {case}")
    print("fp32 readout", case, errs)


# --------------------------------------------------------------------------
# Macroscopic parity over many steps
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kernel,tile", VARIANTS)
def test_smooth_periodic_parity(kernel, tile):
    w = W.random_smooth(300, 37, seed=9, amp=0.1, nsteps=200)
    want = oracle.macro(run_oracle(w))
    with run_gpu(w, Bd.FP64, kernel, tile=tile) as grid:
        assert_parity(grid.macro(), want, linf=1e-12, label="fp64")
    with run_gpu(w, Bd.FP32, kernel, tile=tile) as grid:
        errs = assert_parity(grid.macro(), want, linf=1e-5, l1=1e-5, label="fp32")
    print("fp32 smooth 300x37 200 steps", kernel, tile, errs)


def test_sod_tube_parity():
    """Sod shock tube, 400 x 4, gamma 1.4, Pr 0.71, CFL 0.1, 2000 steps."""
    w = W.sod_tube()
    want = oracle.macro(run_oracle(w))
    with run_gpu(w, Bd.FP64) as grid:
        assert_parity(grid.macro(), want, linf=1e-10, label="fp64")
    with run_gpu(w, Bd.FP32) as grid:
        errs = assert_parity(grid.macro(), want, l1=1e-4, label="fp32")
    print("fp32 sod", errs)


@pytest.fixture(scope="module")
def strong_shock_oracle():
    w = W.strong_shock()           # 2048 x 8, 10000 steps
    return w, oracle.macro(run_oracle(w))


@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
def test_strong_shock_parity(strong_shock_oracle, prec):
    """(rho, u, p) = (5, 0, 100) | (1, 0, 1), 2048 x 8, Pr 1, CFL 0.05,
    10000 steps: parity with the oracle and the exact shock position."""
    w, want = strong_shock_oracle
    with run_gpu(w, prec) as grid:
        got = grid.macro()
        tot = grid.totals()
    if prec == Bd.FP64:
        errs = assert_parity(got, want, linf=1e-9, label="fp64")
    else:
        errs = assert_parity(got, want, l1=1e-4, label="fp32")
    print("strong shock", prec, errs)
    L, R = w.extra["left"], w.extra["right"]
    st = riemann.star_state(L, R, w.gamma)
    x = (np.arange(w.nx) + 0.5) * w.dx
    xs = riemann.shock_position(x, got[0][0], st.rho_r, R[0])
    assert abs(xs - (0.5 + st.shock_r * w.nsteps * w.dt)) < 2 * w.dx
    assert np.all(np.isfinite(tot))


def test_kelvin_helmholtz_reduced_parity():
    w = W.kelvin_helmholtz(n=256, nsteps=1000)
    want = oracle.macro(run_oracle(w))
    with run_gpu(w, Bd.FP32) as grid:
        errs = assert_parity(grid.macro(), want, linf=1e-5, l1=1e-5, label="kh fp32")
    print("fp32 kh 256^2 1000 steps", errs)


def test_vortex_parity():
    w = W.smooth_vortex(n=128, nsteps=500)
    want = oracle.macro(run_oracle(w))
    with run_gpu(w, Bd.FP32) as grid:
        errs = assert_parity(grid.macro(), want, linf=1e-5, l1=1e-5, label="vortex fp32")
    print("fp32 vortex 128^2 500 steps", errs)
    with run_gpu(w, Bd.FP64) as grid:
        assert_parity(grid.macro(), want, linf=1e-12, label="vortex fp64")


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 5), (129, 3), (127, 130), (257, 9)])
@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 1), (1, 0)])
def test_edge_sizes(nx, ny, bcx, bcy):
    w = W.random_smooth(nx, ny, seed=nx + ny, amp=0.05, bc_x=bcx, bc_y=bcy, nsteps=15)
    want = oracle.macro(run_oracle(w))
    for kernel, tile in VARIANTS:
        with run_gpu(w, Bd.FP64, kernel, tile=tile) as grid:
            assert_parity(grid.macro(), want, linf=1e-12, label=f"fp64 k{kernel} t{tile}")
        with run_gpu(w, Bd.FP32, kernel, tile=tile) as grid:
            assert_parity(grid.macro(), want, linf=1e-5, label=f"fp32 k{kernel} t{tile}")


@pytest.mark.parametrize("case", ["kh", "tube", "vortex", "hot"])
def test_fp32_initial_state_is_the_rounded_fp64_one(case):
    """An FP32 grid forms f^eq = M^-1 fhat^eq in double-float arithmetic
    (about 44 bits); rounded to FP32 it equals the FP32 rounding of the FP64
    grid's f^eq except where that value lies within about 2^-44 of a
    rounding boundary: at most one unit in the last place, in a handful of
    the values.  Host and device fields, several chunks of the upload."""
    w = {"kh": W.kelvin_helmholtz(n=2048, nsteps=0),
         "tube": W.riemann_instances(count=1, seed=4, nx_range=(2000, 2000), ny_choices=(256,), nsteps=0)[0],
         "vortex": W.smooth_vortex(n=512, nsteps=0),
         "hot": W.random_smooth(700, 300, seed=9, amp=0.3, nsteps=0)}[case]
    with run_gpu(w, Bd.FP64, nsteps=0) as g64:
        want = g64.get_f().astype(np.float32)
    with run_gpu(w, Bd.FP32, nsteps=0) as g32:
        got = g32.get_f()
    ulps = np.abs(got.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
    print(case, "values off by one ulp:", int(np.count_nonzero(ulps)), "of", ulps.size)
    assert ulps.max() <= 1
    assert np.count_nonzero(ulps) <= max(4, ulps.size // 100000)


@pytest.mark.parametrize("nx,ny", [(200, 40), (2048, 1101)])
@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
def test_device_inputs_match_host_inputs(nx, ny, prec):
    """Host fields are uploaded and initialised in row chunks (2048 x 1101:
    two chunks, the second shorter) and read back to host memory in row
    chunks; device fields and device readouts take one pass.  The states and
    the fields read back agree bit for bit."""
    import torch
    w = W.random_smooth(nx, ny, seed=3, amp=0.05, nsteps=5)
    with run_gpu(w, prec) as a:
        fa = a.get_f()
        ma = a.macro()
    dev = [torch.tensor(np.ascontiguousarray(v), device="cuda") for v in (w.rho, w.ux, w.uy, w.T)]
    p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, w.s, w.bc_x, w.bc_y, prec)
    with Bd.Grid(p, *dev) as b:
        b.step(5)
        fb = b.get_f()
        mb = [torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda") for _ in range(4)]
        b.macro(mb)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(fa, fb)
    for x, y in zip(ma, mb):
        np.testing.assert_array_equal(x, y.cpu().numpy())

# --------------------------------------------------------------------------
# Conserved totals, checkpoint/resume, health
# --------------------------------------------------------------------------
def test_totals_match_oracle():
    w = W.random_smooth(300, 37, seed=5, amp=0.1, nsteps=30)
    g = run_oracle(w)
    want = oracle.totals(g)
    _, _, _, M, _ = oracle.model()
    absq = np.array([np.sum(np.abs(np.tensordot(M[k], g.f, 1))) * w.dx ** 2 for k in range(4)])
    with run_gpu(w, Bd.FP64) as grid:
        fused = grid.totals()
        grid.set_f(grid.get_f())         # forces the standalone reduction
        alone = grid.totals()
    assert np.all(np.abs(fused - want) <= 1e-13 * absq)
    assert np.all(np.abs(alone - fused) <= 1e-14 * absq)
    with run_gpu(w, Bd.FP32) as grid:
        t32 = grid.totals()
    assert np.all(np.abs(t32 - want) <= 1e-5 * absq)


def test_fp64_gpu_conserves_to_roundoff():
    w = W.random_smooth(300, 37, seed=6, amp=0.1)
    with Bd.Grid.from_workload(w, precision=Bd.FP64) as grid:
        f = grid.get_f()
        _, _, _, M, _ = oracle.model()
        absq = np.array([np.sum(np.abs(np.tensordot(M[k], f, 1))) * w.dx ** 2 for k in range(4)])
        grid.step(1)
        t0 = grid.totals()
        for _ in range(10):
            grid.step(1)
            t = grid.totals()
            assert np.all(np.abs(t - t0) <= 1e-13 * absq)


@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
def test_checkpoint_resume_bit_identical(prec):
    w = W.kelvin_helmholtz(n=192, nsteps=0)
    with Bd.Grid.from_workload(w, precision=prec) as a:
        a.step(7)
        ckpt = a.get_f()
        a.step(9)
        fa = a.get_f()
    with Bd.Grid.from_workload(w, precision=prec) as b:
        b.set_f(ckpt)
        b.step(9)
        fb = b.get_f()
    np.testing.assert_array_equal(fa, fb)


@pytest.mark.parametrize("bad", ["rho", "T"])
def test_nonpositive_initial_state_rejected(bad):
    w = W.uniform(40, 12)
    arr = {k: np.ascontiguousarray(getattr(w, k)).copy() for k in ("rho", "ux", "uy", "T")}
    arr[bad][3, 5] = -0.1
    p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, w.s)
    with pytest.raises(Bd.MrtError) as ei:
        Bd.Grid(p, arr["rho"], arr["ux"], arr["uy"], arr["T"])
    assert ei.value.code == Bd.MRT_EINVAL


def test_health_flag_trips_on_blow_up():
    w = W.random_smooth(64, 16, seed=1, amp=0.2)
    s = np.full(16, 2.5 / w.dt)         # sigma = 2.5 > 1: outside the stable interval
    p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, s, 0, 0, Bd.FP32)
    with Bd.Grid(p, w.rho, w.ux, w.uy, w.T) as g:
        assert g.health() == Bd.MRT_OK
        g.step(400)
        assert g.health() == Bd.MRT_EUNSTABLE
        with pytest.raises(Bd.MrtError):
            g.totals()


# --------------------------------------------------------------------------
# Full size, bench launch configuration: sampled windows
# --------------------------------------------------------------------------
def _window_oracle_step(w, f_full, y0, x0, n):
    """One oracle step on an (n+2)^2 periodic window around [y0:y0+n, x0:x0+n];
    the interior depends only on the window, so it is exact there."""
    ys = (np.arange(y0 - 1, y0 + n + 1)) % w.ny
    xs = (np.arange(x0 - 1, x0 + n + 1)) % w.nx
    fw = np.ascontiguousarray(f_full[:, ys][:, :, xs].astype(np.float64))
    g = oracle.Grid(n + 2, n + 2, w.dx, w.dt, w.b, w.s, oracle.BC_PERIODIC, oracle.BC_PERIODIC)
    g.f = fw
    g.gx = np.zeros((16, 2, n + 2))
    g.gy = np.zeros((16, 2, n + 2))
    return oracle.step(g, fw)[:, 1:-1, 1:-1]


def test_full_size_kh_sampled_windows():
    """4096^2 Kelvin-Helmholtz in FP32 with the TMA kernel (the benchmark's
    configuration): after 3 steps, 12 seeded 48^2 windows (including the
    periodic corners and strip/chunk seams) of step 3 -> 4 match the oracle."""
    w = W.kelvin_helmholtz(n=4096, nsteps=0)
    rng = np.random.default_rng(0)
    n = 48
    corners = [(0, 0), (w.ny - n, w.nx - n), (0, w.nx - n), (w.ny - n, 0), (2000, 128 * 16 - 24)]
    wins = corners + [(int(rng.integers(0, w.ny - n)), int(rng.integers(0, w.nx - n))) for _ in range(7)]
    with Bd.Grid.from_workload(w, precision=Bd.FP32, kernel=Bd.KERNEL_TMA) as grid:
        assert grid.info()["kernel"] == Bd.KERNEL_TMA and grid.info()["tile"] == 6
        grid.step(3)
        f3 = grid.get_f()
        grid.step(1)
        f4 = grid.get_f()
        tot = grid.totals()
    for (y0, x0) in wins:
        want = _window_oracle_step(w, f3, y0, x0, n)
        got = f4[:, y0:y0 + n, x0:x0 + n].astype(np.float64)
        scale = np.max(np.abs(want))
        assert np.max(np.abs(got - want)) <= 2e-6 * scale, (y0, x0)
    assert np.all(np.isfinite(tot)) and abs(tot[0] - 1.0) < 1e-6


def test_automatic_kernel_and_tile_choice():
    """Tile 0 / MRT_KERNEL_AUTO: the work-queue tile 6 on grids with at least
    two 8-row items per resident CTA, the static tile 4 (FP32) or 1 (FP64)
    on smaller ones, the direct kernel on small FP64 grids and the split
    kernel on tiny ones (8192 cells in FP64, 2048 in FP32)."""
    cases = [(W.kelvin_helmholtz(n=2048, nsteps=0), Bd.FP32, (Bd.KERNEL_TMA, 6)),
             (W.kelvin_helmholtz(n=2048, nsteps=0), Bd.FP64, (Bd.KERNEL_TMA, 6)),
             (W.kelvin_helmholtz(n=512, nsteps=0), Bd.FP32, (Bd.KERNEL_TMA, 4)),
             (W.kelvin_helmholtz(n=512, nsteps=0), Bd.FP64, (Bd.KERNEL_TMA, 1)),
             (W.sod_tube(), Bd.FP64, (Bd.KERNEL_SPLIT, None)),
             (W.sod_tube(), Bd.FP32, (Bd.KERNEL_SPLIT, None)),
             (W.colliding_shocks(), Bd.FP64, (Bd.KERNEL_SPLIT, None)),
             (W.colliding_shocks(), Bd.FP32, (Bd.KERNEL_TMA, 4)),
             (W.strong_shock(), Bd.FP64, (Bd.KERNEL_DIRECT, None)),
             (W.strong_shock(), Bd.FP32, (Bd.KERNEL_TMA, 4))]
    for w, prec, (kernel, tile) in cases:
        with Bd.Grid.from_workload(w, precision=prec) as g:
            info = g.info()
        assert info["kernel"] == kernel, (w.name, prec, info)
        if tile is not None:
            assert info["tile"] == tile, (w.name, prec, info)


@pytest.mark.parametrize("bcy", [Bd.BC_PERIODIC, Bd.BC_FIXED_EQ, Bd.BC_REFLECT_FIXED])
def test_reflecting_wall_parity(bcy):
    """Reflecting wall at the low x end (fixed inflow at the high end), and
    on y as well in the last case: every kernel variant against the oracle,
    300 x 37 (three strips, a ragged tail), 15 steps."""
    w = W.random_smooth(300, 37, seed=23, amp=0.1, bc_x=Bd.BC_REFLECT_FIXED, bc_y=bcy, nsteps=15)
    want = oracle.macro(run_oracle(w))
    for kernel, tile in VARIANTS:
        with run_gpu(w, Bd.FP64, kernel, tile=tile) as grid:
            assert_parity(grid.macro(), want, linf=1e-12, label=f"fp64 k{kernel} t{tile}")
        with run_gpu(w, Bd.FP32, kernel, tile=tile) as grid:
            assert_parity(grid.macro(), want, linf=1e-5, label=f"fp32 k{kernel} t{tile}")


def test_reflecting_wall_resume():
    """mrt_set_f refreshes the wall's ghost from the new state (resume is bit
    identical)."""
    w = W.random_smooth(140, 21, seed=4, amp=0.1, bc_x=Bd.BC_REFLECT_FIXED, bc_y=Bd.BC_REFLECT_FIXED, nsteps=0)
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as a:
        a.step(5)
        ck = a.get_f()
        a.step(6)
        want = a.get_f()
        a.set_f(np.zeros_like(ck) + 1.0)      # disturb the ghosts' sources
        a.set_f(ck)
        a.step(6)
        np.testing.assert_array_equal(a.get_f(), want)


def test_grids_on_concurrent_streams():
    """Two grids stepped with interleaved launches on their own streams
    (each with its own work-queue counters) give the same states, bit for
    bit, as each stepped alone."""
    import torch
    wa = W.kelvin_helmholtz(n=2048, nsteps=0, seed=1)
    wb = W.random_smooth(700, 300, seed=2, amp=0.1)
    alone = []
    for w, prec in ((wa, Bd.FP32), (wb, Bd.FP64)):
        with Bd.Grid.from_workload(w, precision=prec) as g:
            g.step(9)
            alone.append(g.get_f())
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    ga = Bd.Grid.from_workload(wa, precision=Bd.FP32, stream=sa.cuda_stream)
    gb = Bd.Grid.from_workload(wb, precision=Bd.FP64, stream=sb.cuda_stream)
    try:
        assert ga.info()["tile"] == 6
        for _ in range(3):
            ga.step(3)
            gb.step(3)
        np.testing.assert_array_equal(ga.get_f(), alone[0])
        np.testing.assert_array_equal(gb.get_f(), alone[1])
    finally:
        ga.close()
        gb.close()


@pytest.mark.parametrize("kernel,tile", [(Bd.KERNEL_TMA, 4), (Bd.KERNEL_TMA, 6), (Bd.KERNEL_DIRECT, 0)])
@pytest.mark.parametrize("prec", [Bd.FP32, Bd.FP64])
def test_graph_replayed_steps_match_single_steps(kernel, tile, prec):
    """mrt_step(n) replays two-step CUDA graphs for all but its last step;
    the states are bit for bit those of n calls of one step each (every
    step launched directly), for odd and even n, and after a reverse-mode
    run has shifted the work-queue counter parity against the buffer index
    (a graph is kept per starting state)."""
    w = W.random_smooth(700, 150, seed=11, amp=0.1, bc_x=Bd.BC_FIXED_EQ)
    with Bd.Grid.from_workload(w, precision=prec, kernel=kernel, tile=tile) as a, \
            Bd.Grid.from_workload(w, precision=prec, kernel=kernel, tile=tile) as b:
        for n in (7, 6, 5):
            a.step(n)
            for _ in range(n):
                b.step(1)
            np.testing.assert_array_equal(a.get_f(), b.get_f())
            np.testing.assert_array_equal(a.totals(), b.totals())
        f = a.get_f()
        for g in (a, b):
            # the record's steps move cur and the parity together; the
            # backward's segment recompute moves the parity alone
            g.adjoint_record(w.rho, w.ux, w.uy, w.T, 3, 2)
            g.adjoint_backward(np.full((w.ny, w.nx), w.dx * w.dx))
            g.set_f(f)
        a.step(9)
        for _ in range(9):
            b.step(1)
        np.testing.assert_array_equal(a.get_f(), b.get_f())
        assert a.health() == Bd.MRT_OK and a.info()["steps"] == b.info()["steps"]


@pytest.mark.parametrize("prec,tol", [(Bd.FP64, 1e-12), (Bd.FP32, 1e-6)])
def test_direct_kernel_totals_with_multi_row_blocks(prec, tol):
    """The direct kernel runs 32 x BY blocks (BY up to 8); the totals its
    last step reduces match the oracle's totals of the same state (a block
    reduction that took warps from threadIdx.x alone summed one warp of
    each block and stale shared memory)."""
    for nx, ny in ((700, 150), (360, 100)):
        w = W.random_smooth(nx, ny, seed=5, amp=0.1)
        g = run_oracle(w, 3)
        want = oracle.totals(g)
        _, _, _, M, _ = oracle.model()
        scale = np.array([np.sum(np.abs(np.tensordot(M[k], g.f, 1))) * w.dx ** 2 for k in range(4)])
        with run_gpu(w, prec, Bd.KERNEL_DIRECT, nsteps=3) as grid:
            got = grid.totals()
        assert np.all(np.abs(got - want) <= tol * scale), (nx, ny, got, want)


@pytest.mark.parametrize("tile", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("prec,tol", [(Bd.FP64, 1e-13), (Bd.FP32, 1e-6)])
def test_tma_totals_fold_row_runs(tile, prec, tol):
    """The strip kernels sum each column's 16 outputs over runs of at most 8
    rows and fold the conserved moments of those sums into the totals; on
    row bands and items whose heights are not multiples of 8 (150 rows,
    ragged last strip) the fused totals match the oracle's totals of the
    same state."""
    w = W.random_smooth(700, 150, seed=8, amp=0.1, bc_x=Bd.BC_FIXED_EQ)
    g = run_oracle(w, 3)
    want = oracle.totals(g)
    _, _, _, M, _ = oracle.model()
    scale = np.array([np.sum(np.abs(np.tensordot(M[k], g.f, 1))) * w.dx ** 2 for k in range(4)])
    with Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_TMA, tile=tile) as grid:
        grid.step(3)
        got = grid.totals()
        assert grid.info()["tile"] == tile
    assert np.all(np.abs(got - want) <= tol * scale), (tile, got, want)
