"""GPU reverse mode against the oracle's reverse mode and finite differences.

Tolerances: FP64 GPU vs oracle 1e-10 relative (L2 over each gradient field;
only summation order differs); FP32 GPU vs FP64 oracle 1e-3 relative L2;
finite differences (central, h = 1e-4) to 1e-4 relative plus an absolute
floor for directions whose gradient vanishes by symmetry.
"""
import numpy as np
import pytest

import oracle
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


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("prec,tol", [(Bd.FP64, 1e-12), (Bd.FP32, 2e-5)])
@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 2)])
def test_adjoint_step_matches_oracle(prec, tol, bcx, bcy):
    w = W.random_smooth(140, 21, seed=8, amp=0.1, bc_x=bcx, bc_y=bcy)
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    f = oracle.step(g)
    rng = np.random.default_rng(3)
    lam_next = rng.standard_normal(f.shape)
    dt = np.float64 if prec == Bd.FP64 else np.float32
    f_in, l_in = f.astype(dt), lam_next.astype(dt)
    gs = np.zeros(16)
    want = oracle.step_adjoint(g, f_in.astype(np.float64), l_in.astype(np.float64), np.zeros_like(g.gx),
                               np.zeros_like(g.gy), gs)
    with Bd.Grid.from_workload(w, precision=prec) as grid:
        got, gs_gpu = grid.adjoint_step(f_in, l_in)
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    assert np.all(gs_gpu[:4] == 0)
    np.testing.assert_allclose(gs_gpu[4:], gs[4:], rtol=tol * 50, atol=tol * np.max(np.abs(gs)))


def _loss(target, dx):
    def lg(r):
        d = r - target
        return 0.5 * np.sum(d * d) * dx * dx, d * dx * dx
    return lg


def _gpu_grads(w, prec, nsteps, ckpt, lg, kernel=Bd.KERNEL_AUTO, dL=None):
    """Loss and gradients; dL overrides the upstream gradient dL/drho_N."""
    with Bd.Grid.from_workload(w, precision=prec, kernel=kernel) as grid:
        grid.adjoint_record(w.rho, w.ux, w.uy, w.T, nsteps, ckpt)
        rhoN = grid.macro()[0]
        L, dL_own = lg(rhoN)
        out = grid.adjoint_backward(dL_own if dL is None else dL)
    return L, out


@pytest.mark.parametrize("case", ["vortex", "tube", "wall"])
def test_adjoint_run_matches_oracle(case):
    if case == "vortex":
        w = W.smooth_vortex(n=40, nsteps=30, r0=0.15)
        target = W.vortex_target(w)
    elif case == "tube":
        w = W.sod_tube(nx=150, ny=5, nsteps=30)
        target = w.rho * 0.97 + 0.01
    else:
        # reflecting walls at the low ends of both axes, inflow at the high ends
        w = W.random_smooth(150, 37, seed=31, amp=0.1, bc_x=Bd.BC_REFLECT_FIXED, bc_y=Bd.BC_REFLECT_FIXED,
                            nsteps=30)
        target = w.rho * 0.98 + 0.02
    lg = _loss(target, w.dx)
    ref = oracle.adjoint_run(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.nsteps, lg,
                             w.bc_x, w.bc_y, ckpt=7)
    for prec, tol in ((Bd.FP64, 1e-10), (Bd.FP32, 1e-3)):
        for kernel in (Bd.KERNEL_TMA, Bd.KERNEL_DIRECT):
            L, got = _gpu_grads(w, prec, w.nsteps, 7, lg, kernel)
            assert abs(L - ref[0]) <= (1e-12 if prec == Bd.FP64 else 1e-5) * abs(ref[0])
            for name, a, b in zip(("rho", "ux", "uy", "T"), got[:4], ref[1:5]):
                # fields whose gradient vanishes by symmetry are compared to the largest one
                scale = max(np.linalg.norm(b), 1e-4 * max(np.linalg.norm(x) for x in ref[1:5]))
                err = np.linalg.norm(a - b) / scale
                assert err <= tol, (case, prec, kernel, name, err)
            gs, gref = got[4], ref[5]
            assert np.all(gs[:4] == 0)
            err = np.linalg.norm(gs - gref) / np.linalg.norm(gref)
            assert err <= tol, (case, prec, kernel, "rates", err)


def test_checkpoint_interval_does_not_change_gradients():
    w = W.smooth_vortex(n=48, nsteps=25, r0=0.15)
    lg = _loss(W.vortex_target(w), w.dx)
    _, a = _gpu_grads(w, Bd.FP64, w.nsteps, 25, lg)
    _, b = _gpu_grads(w, Bd.FP64, w.nsteps, 4, lg)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_full_size_vortex_adjoint_against_finite_differences():
    """The 512^2 smooth-vortex configuration (Ma 0.8, gamma 1.4, Pr 0.71),
    500 steps, checkpoints every 50: FP64 GPU gradient against central
    differences of the FP64 GPU loss (h = 1e-4), and the FP32 GPU gradient
    against the FP64 one."""
    w = W.smooth_vortex(n=512, nsteps=500)
    lg = _loss(W.vortex_target(w), w.dx)
    L64, g64 = _gpu_grads(w, Bd.FP64, 500, 50, lg)
    with Bd.Grid.from_workload(w, precision=Bd.FP64) as grid:
        grid.step(500)
        dL64 = lg(grid.macro()[0])[1]
    # FP32 reverse sweep fed the same upstream gradient as the FP64 run
    _, g32s = _gpu_grads(w, Bd.FP32, 500, 50, lg, dL=dL64)
    for a, b in zip(g32s, g64):
        assert _rel(a, b) <= 1e-3
    # End to end in FP32: rho_N itself carries the FP32 rounding of f^0
    # (about 1e-7 of rho), which enters dL/drho_N = (rho_N - rho_tgt) dx^2 in
    # every cell, far from the vortex too; that bounds the agreement at ~5e-3.
    L32, g32 = _gpu_grads(w, Bd.FP32, 500, 50, lg)
    assert abs(L32 - L64) <= 1e-4 * abs(L64)
    for a, b in zip(g32, g64):
        assert _rel(a, b) <= 5e-3

    def loss_of(**kw):
        a = dict(rho=w.rho, ux=w.ux, uy=w.uy, T=w.T, s=w.s)
        a.update(kw)
        p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, a["s"], w.bc_x, w.bc_y, Bd.FP64)
        with Bd.Grid(p, a["rho"], a["ux"], a["uy"], a["T"]) as grid:
            grid.step(500)
            return lg(grid.macro()[0])[0]

    h = 1e-4
    rng = np.random.default_rng(11)
    for name, base, grad in (("rho", w.rho, g64[0]), ("ux", w.ux, g64[1]), ("uy", w.uy, g64[2]),
                             ("T", w.T, g64[3])):
        d = rng.standard_normal(base.shape)
        fd = (loss_of(**{name: base + h * d}) - loss_of(**{name: base - h * d})) / (2 * h)
        got = np.sum(grad * d)
        assert abs(got - fd) <= 1e-4 * abs(fd) + 1e-6 * np.sum(np.abs(grad)) * h, (name, got, fd)
    for k in (4, 5, 7, 9, 13):
        sp, sm = w.s.copy(), w.s.copy()
        sp[k] *= 1 + h
        sm[k] *= 1 - h
        fd = (loss_of(s=sp) - loss_of(s=sm)) / (2 * h)
        got = g64[4][k] * w.s[k]
        assert abs(got - fd) <= 1e-4 * abs(fd) + 1e-6 * np.max(np.abs(g64[4] * w.s)), (k, got, fd)


def test_autograd_function_matches_adjoint():
    import torch

    from paper_1004_5442_gb300.autograd import mrt_run
    w = W.smooth_vortex(n=64, nsteps=40, r0=0.15)
    target = torch.tensor(W.vortex_target(w), device="cuda")
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda", requires_grad=True)
    rho0, ux0, uy0, T0 = dev(w.rho), dev(w.ux), dev(w.uy), dev(w.T)
    s = torch.tensor(w.s, device="cuda", requires_grad=True)
    params = dict(nx=w.nx, ny=w.ny, dx=w.dx, dt=w.dt, gamma=w.gamma, precision=Bd.FP64)
    rhoN = mrt_run(rho0, ux0, uy0, T0, s, params, w.nsteps, 10)
    L = 0.5 * torch.sum((rhoN - target) ** 2) * w.dx ** 2
    L.backward()
    lg = _loss(target.cpu().numpy(), w.dx)
    _, ref = _gpu_grads(w, Bd.FP64, w.nsteps, 10, lg)
    for t, r in zip((rho0, ux0, uy0, T0), ref[:4]):
        np.testing.assert_allclose(t.grad.cpu().numpy(), r, rtol=1e-12, atol=1e-14 * np.max(np.abs(r)))
    np.testing.assert_allclose(s.grad.cpu().numpy(), ref[4], rtol=1e-12, atol=0)


def test_autograd_second_backward():
    """retain_graph=True keeps the recorded run: a second backward gives the
    same gradients bit for bit (accumulated twice in .grad); without it a
    second backward raises PyTorch's error.  Run on a side stream, so the
    reverse sweep must wait for the caller's stream by event."""
    import torch

    from paper_1004_5442_gb300.autograd import mrt_run
    w = W.smooth_vortex(n=48, nsteps=20, r0=0.15)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        target = torch.tensor(W.vortex_target(w), device="cuda")
        dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda", requires_grad=True)
        rho0, ux0, uy0, T0 = dev(w.rho), dev(w.ux), dev(w.uy), dev(w.T)
        s = torch.tensor(w.s, device="cuda", requires_grad=True)
        params = dict(nx=w.nx, ny=w.ny, dx=w.dx, dt=w.dt, gamma=w.gamma, precision=Bd.FP64)
        rhoN = mrt_run(rho0, ux0, uy0, T0, s, params, w.nsteps, 5)
        L = 0.5 * torch.sum((rhoN - target) ** 2) * w.dx ** 2
        L.backward(retain_graph=True)
        first = [t.grad.clone() for t in (rho0, ux0, uy0, T0, s)]
        L.backward(retain_graph=True)
        for t, g1 in zip((rho0, ux0, uy0, T0, s), first):
            assert torch.equal(t.grad, 2 * g1)
        L.backward()
        with pytest.raises(RuntimeError):
            L.backward()
    side.synchronize()
