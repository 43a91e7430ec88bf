"""Pins of the oracle's reverse mode (gradients of a loss of rho_N with
respect to the initial fields and the 16 relaxation rates): complex-step
equilibrium Jacobian against finite differences, the per-step transpose
against a finite-difference tangent (dot-product test), whole-run gradients
against central finite differences (h = 1e-4, absolute for fields, relative
for rates), and dL/ds_1..4 = 0."""
import numpy as np
import pytest

from paper_1004_5442_gb300 import workloads as W


def test_feq_jacobian_complex_step(orc):
    b = orc.b_of_gamma(1.4)
    rng = np.random.default_rng(0)
    for _ in range(5):
        rho = rng.uniform(0.5, 3)
        jx, jy = rng.uniform(-1, 1, 2) * rho
        e = b * rho * rng.uniform(0.5, 3) + (jx * jx + jy * jy) / rho
        m = np.array([rho, jx, jy, e])
        J = orc.feq_jacobian(*m, b)
        np.testing.assert_allclose(orc.feq_moments_via_cplx(*m, b), orc.feq_moments(*m, b), rtol=1e-14,
                                   atol=1e-14)
        for j in range(4):
            h = 1e-6 * max(abs(m[j]), 1.0)
            mp, mm = m.copy(), m.copy()
            mp[j] += h
            mm[j] -= h
            fd = (orc.feq_moments(*mp, b) - orc.feq_moments(*mm, b)) / (2 * h)
            np.testing.assert_allclose(J[:, j], fd, rtol=1e-6, atol=1e-8 * np.max(np.abs(fd)))
    # conserved rows are the identity
    np.testing.assert_array_equal(J[:4], np.eye(4))


@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 2), (1, 2)])
def test_step_transpose_dot_product(orc, bcx, bcy):
    w = W.random_smooth(9, 7, seed=2, amp=0.1, bc_x=bcx, bc_y=bcy)
    g = orc.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    rng = np.random.default_rng(1)
    f = g.f * (1 + 0.01 * rng.standard_normal(g.f.shape))
    d = rng.standard_normal(f.shape)
    lam = rng.standard_normal(f.shape)
    h = 1e-6
    tangent = (orc.step(g, f + h * d) - orc.step(g, f - h * d)) / (2 * h)
    gxb, gyb, gs = np.zeros_like(g.gx), np.zeros_like(g.gy), np.zeros(16)
    adj = orc.step_adjoint(g, f, lam, gxb, gyb, gs)
    lhs = np.sum(lam * tangent)
    rhs = np.sum(adj * d)
    assert abs(lhs - rhs) <= 1e-8 * np.sum(np.abs(lam * tangent))
    # ghost adjoint against a perturbation of the ghost values (the
    # reflecting wall's ghost is not a free value: its adjoint goes to the
    # mirrored cell, covered by the dot product above; the inflow end of a
    # walled axis is a fixed ghost like the others)
    if bcx in (1, 2):
        dg = rng.standard_normal(g.gx.shape)
        gp, gm = g.gx + h * dg, g.gx - h * dg
        g.gx = gp
        fp = orc.step(g, f)
        g.gx = gm
        fm = orc.step(g, f)
        t = np.sum(lam * (fp - fm) / (2 * h))
        assert abs(t - np.sum(gxb * dg)) <= 1e-8 * max(abs(t), 1e-300) + 1e-12
        if bcx == 2:
            assert np.all(gxb[:, 0, :] == 0.0)


def _loss(target, dx):
    def lg(r):
        d = r - target
        return 0.5 * np.sum(d * d) * dx * dx, d * dx * dx
    return lg


@pytest.mark.parametrize("case", ["vortex", "tube", "wall"])
def test_adjoint_matches_finite_differences(orc, case):
    if case == "vortex":
        w = W.smooth_vortex(n=20, nsteps=24, r0=0.15)
        target = W.vortex_target(w)
    elif case == "tube":
        w = W.sod_tube(nx=40, ny=3, nsteps=30)
        target = w.rho * 0.97 + 0.01
    else:
        # reflecting wall on the left, inflow on the right, wall in y too
        w = W.random_smooth(20, 9, seed=31, amp=0.1, bc_x=orc.BC_REFLECT_FIXED, bc_y=orc.BC_REFLECT_FIXED,
                            nsteps=24)
        target = w.rho * 0.98 + 0.02
    lg = _loss(target, w.dx)
    args = (w.nx, w.ny, w.dx, w.dt, w.b)
    L, gr, gu, gv, gT, gs = orc.adjoint_run(*args, w.s, w.rho, w.ux, w.uy, w.T, w.nsteps, lg,
                                            w.bc_x, w.bc_y, ckpt=7)
    assert np.all(gs[:4] == 0.0)

    def fl(s=w.s, rho=w.rho, ux=w.ux, uy=w.uy, T=w.T):
        return orc.forward_loss(*args, s, rho, ux, uy, T, w.nsteps, lg, w.bc_x, w.bc_y)

    h = 1e-4
    gscale = np.max(np.abs(gs * w.s))
    for k in range(4, 16):
        sp, sm = w.s.copy(), w.s.copy()
        sp[k] *= 1 + h
        sm[k] *= 1 - h
        fd = (fl(s=sp) - fl(s=sm)) / (2 * h)      # = s_k dL/ds_k
        assert abs(fd - gs[k] * w.s[k]) <= 1e-5 * gscale + 1e-4 * abs(fd), k
    rng = np.random.default_rng(5)
    # scale for fields whose gradient vanishes by symmetry (then FD is O(h^2))
    gabs = max(np.sum(np.abs(a)) for a in (gr, gu, gv, gT))
    for name, base, grad in (("rho", w.rho, gr), ("ux", w.ux, gu), ("uy", w.uy, gv), ("T", w.T, gT)):
        for _ in range(2):
            d = rng.standard_normal(base.shape)
            fd = (fl(**{name: base + h * d}) - fl(**{name: base - h * d})) / (2 * h)
            got = np.sum(grad * d)
            assert abs(got - fd) <= 1e-4 * abs(fd) + 1e-6 * gabs, (name, got, fd)
        # single entries
        for _ in range(2):
            iy, ix = rng.integers(0, w.ny), rng.integers(0, w.nx)
            d = np.zeros_like(base)
            d[iy, ix] = 1.0
            fd = (fl(**{name: base + h * d}) - fl(**{name: base - h * d})) / (2 * h)
            got = grad[iy, ix]
            assert abs(got - fd) <= 1e-4 * abs(fd) + 1e-6 * gabs, (name, iy, ix, got, fd)


def test_checkpointing_does_not_change_the_gradient(orc):
    w = W.smooth_vortex(n=16, nsteps=20, r0=0.15)
    lg = _loss(W.vortex_target(w), w.dx)
    args = (w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.nsteps, lg)
    a = orc.adjoint_run(*args, ckpt=None)
    b = orc.adjoint_run(*args, ckpt=3)
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(x, y)
