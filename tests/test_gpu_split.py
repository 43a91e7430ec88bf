"""The split kernel (MRT_KERNEL_SPLIT: four warps per 32-cell row segment,
one per velocity group) runs the phases of the cell update across the warps
with the arithmetic of the one-thread-per-cell direct kernel, so the two
agree to rounding: every boundary kind, both precisions, both advection
operators, grids with a ragged last segment and the 3 x 3 minimum.  A call
of two or more steps runs them all in one cooperative launch (tiles wait for
their neighbours' previous step through per-tile counters); its states agree
with those of single-step calls to rounding, odd and even counts.  Totals agree to rounding, the guard band stays clean, the health
flag trips, the reverse mode of a split grid matches the direct grid's, and
the oracle agrees as for the other kernels."""
import numpy as np
import pytest

import oracle
from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W
from _parity import assert_parity, run_oracle

pytestmark = pytest.mark.gpu

BCS = [(Bd.BC_PERIODIC, Bd.BC_PERIODIC), (Bd.BC_FIXED_EQ, Bd.BC_PERIODIC), (Bd.BC_PERIODIC, Bd.BC_FIXED_EQ),
       (Bd.BC_REFLECT_FIXED, Bd.BC_PERIODIC), (Bd.BC_REFLECT_FIXED, Bd.BC_REFLECT_FIXED),
       (Bd.BC_FIXED_EQ, Bd.BC_FIXED_EQ)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    yield


def _run(w, prec, kernel, nsteps, adv):
    with Bd.Grid.from_workload(w, precision=prec, kernel=kernel, advection=adv) as g:
        g.step(nsteps)
        assert g.info()["kernel"] == kernel
        return g.get_f(), g.totals(), g.debug_padding()


@pytest.mark.parametrize("adv", [Bd.ADV_LW, Bd.ADV_LW2D])
@pytest.mark.parametrize("prec", [Bd.FP64, Bd.FP32])
@pytest.mark.parametrize("bcx,bcy", BCS)
def test_split_against_direct(bcx, bcy, prec, adv):
    tol = 1e-13 if prec == Bd.FP64 else 2e-6
    for nx, ny, steps in ((300, 37, 7), (64, 5, 4), (3, 3, 5), (1300, 4, 12)):
        w = W.random_smooth(nx, ny, seed=nx + ny, amp=0.1, bc_x=bcx, bc_y=bcy)
        fs, ts, pad = _run(w, prec, Bd.KERNEL_SPLIT, steps, adv)
        fd, td, _ = _run(w, prec, Bd.KERNEL_DIRECT, steps, adv)
        scale = np.max(np.abs(fd))
        assert np.max(np.abs(fs - fd)) <= tol * scale, (nx, ny, np.max(np.abs(fs - fd)) / scale)
        assert pad == 0
        _, _, _, M, _ = oracle.model()
        tscale = np.array([np.sum(np.abs(np.tensordot(M[k], fd.astype(np.float64), 1))) for k in range(4)]) * w.dx ** 2
        assert np.all(np.abs(ts - td) <= tol * tscale), (nx, ny, ts, td)


@pytest.mark.parametrize("adv", [Bd.ADV_LW, Bd.ADV_LW2D])
@pytest.mark.parametrize("prec", [Bd.FP64, Bd.FP32])
@pytest.mark.parametrize("bcx,bcy", [BCS[0], BCS[3], BCS[5]])
def test_multi_step_launch_equals_single_steps(bcx, bcy, prec, adv):
    """step(n) with n >= 2 is one cooperative launch; n calls of step(1) are
    n launches of the one-tile-per-block kernel.  Both run split_tile, but
    the compiler chooses multiply-add contractions per kernel, so the states
    agree to rounding (1e-13 of max |f| in FP64, 2e-6 in FP32 after at most
    16 steps), as do the totals; a missed wait or a stale read would differ
    by orders of magnitude more."""
    for nx, ny, steps in ((300, 37, 9), (1300, 4, 16), (40, 3, 2), (700, 150, 5)):
        w = W.random_smooth(nx, ny, seed=3 * nx + ny, amp=0.1, bc_x=bcx, bc_y=bcy)
        with Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_SPLIT, advection=adv) as a, \
                Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_SPLIT, advection=adv) as b:
            a.step(steps)
            for _ in range(steps):
                b.step(1)
            fa, fb = a.get_f(), b.get_f()
            tol = 1e-13 if prec == Bd.FP64 else 2e-6
            assert np.max(np.abs(fa - fb)) <= tol * np.max(np.abs(fb)), (nx, ny, np.max(np.abs(fa - fb)))
            ta, tb = a.totals(), b.totals()
            assert np.all(np.abs(ta - tb) <= tol * np.max(np.abs(tb))), (nx, ny, ta, tb)
            assert a.info()["steps"] == steps and a.health() == Bd.MRT_OK and a.debug_padding() == 0


@pytest.mark.parametrize("prec,tol", [(Bd.FP64, 1e-12), (Bd.FP32, 2e-5)])
def test_split_against_oracle(prec, tol):
    w = W.sod_tube(nx=400, ny=4, nsteps=200)
    want = oracle.macro(run_oracle(w))
    with Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_SPLIT) as g:
        g.step(w.nsteps)
        assert_parity(g.macro(), want, linf=tol, label="split")
        assert g.health() == Bd.MRT_OK


@pytest.mark.parametrize("prec", [Bd.FP64, Bd.FP32])
def test_split_health_flag(prec):
    w = W.random_smooth(64, 16, seed=1, amp=0.2)
    s = np.full(16, 2.5 / w.dt)         # sigma = 2.5 > 1: outside the stable interval
    p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, s, 0, 0, prec, 0.0, Bd.KERNEL_SPLIT)
    with Bd.Grid(p, w.rho, w.ux, w.uy, w.T) as g:
        assert g.health() == Bd.MRT_OK
        g.step(400)
        assert g.health() == Bd.MRT_EUNSTABLE


def test_split_reverse_mode_matches_direct():
    w = W.smooth_vortex(n=40, nsteps=12, r0=0.15)
    dL = np.random.default_rng(2).standard_normal((w.ny, w.nx)) * w.dx ** 2
    out = {}
    for kernel in (Bd.KERNEL_SPLIT, Bd.KERNEL_DIRECT):
        with Bd.Grid.from_workload(w, precision=Bd.FP64, kernel=kernel) as g:
            g.adjoint_record(w.rho, w.ux, w.uy, w.T, w.nsteps, 5)
            out[kernel] = g.adjoint_backward(dL)
    # the recorded forward states agree to rounding, so do the gradients (the
    # rate gradients are sums over the run with cancellation: 1e-9 of their norm)
    for a, b in zip(out[Bd.KERNEL_SPLIT], out[Bd.KERNEL_DIRECT]):
        assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(b)
