"""Pins of the oracle's time step: fixed points, conservation, flux balance,
symmetry, the BGK limit, the Lax-Wendroff amplification factor, and an
independent dense numpy evaluation on a tiny grid."""
import numpy as np
import pytest

from paper_1004_5442_gb300 import workloads as W


def _grid(orc, w, s=None):
    return orc.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s if s is None else s,
                      w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)


@pytest.mark.parametrize("bcx", [W.BC_PERIODIC, W.BC_FIXED_EQ])
@pytest.mark.parametrize("state", [(1, 0, 0, 1), (5, 0.3, -0.2, 20), (0.125, 1.5, 0.5, 0.8)])
def test_uniform_equilibrium_is_fixed_point(orc, bcx, state):
    rho, ux, uy, T = state
    w = W.uniform(9, 7, rho=rho, ux=ux, uy=uy, T=T, bc_x=bcx, bc_y=W.BC_FIXED_EQ)
    g = _grid(orc, w)
    f1 = orc.step(g)
    assert np.max(np.abs(f1 - g.f)) <= 1e-13 * np.max(np.abs(g.f))


def test_conservation_periodic(orc):
    """rho, j, e are collision invariants (fhat_1..4 = fhat^eq_1..4) and the
    periodic LW fluxes telescope: totals are constant to round-off."""
    w = W.random_smooth(24, 20, seed=3, amp=0.1)
    g = _grid(orc, w)
    _, _, _, M, _ = orc.model()
    t0 = orc.totals(g)
    abs_scale = np.array([np.sum(np.abs(np.tensordot(M[k], g.f, 1))) * w.dx ** 2 for k in range(4)])
    for _ in range(20):
        orc.run(g, 1)
        t = orc.totals(g)
        assert np.all(np.abs(t - t0) <= 1e-13 * abs_scale), (t - t0) / abs_scale


def test_tube_flux_balance(orc):
    """Fixed-equilibrium ends with the initial states at rest: per step mass
    and energy are unchanged and the x momentum gains dt (P_L - P_R) ny dx
    (telescoped LW fluxes), while the waves are inside the domain."""
    w = W.sod_tube(nx=200, ny=4)
    g = _grid(orc, w)
    t_prev = orc.totals(g)
    PL, PR = 1.0, 0.1
    for _ in range(60):
        orc.run(g, 1)
        t = orc.totals(g)
        d = t - t_prev
        assert abs(d[0]) < 1e-13 * t[0]
        assert abs(d[3]) < 1e-13 * t[3]
        assert abs(d[2]) < 1e-15
        want = w.dt * (PL - PR) * w.ny * w.dx
        assert abs(d[1] - want) < 1e-10 * want
        t_prev = t


def test_mirror_symmetry(orc):
    w = W.random_smooth(16, 12, seed=7, amp=0.1, bc_x=W.BC_FIXED_EQ)
    g = _grid(orc, w)
    wm = W.Workload(**{**w.__dict__})
    wm.rho, wm.T, wm.uy = w.rho[:, ::-1].copy(), w.T[:, ::-1].copy(), w.uy[:, ::-1].copy()
    wm.ux = -w.ux[:, ::-1].copy()
    gm = _grid(orc, wm)
    orc.run(g, 25)
    orc.run(gm, 25)
    r, u, v, T = orc.macro(g)
    rm, um, vm, Tm = orc.macro(gm)
    np.testing.assert_allclose(rm[:, ::-1], r, rtol=1e-12)
    np.testing.assert_allclose(-um[:, ::-1], u, atol=1e-12)
    np.testing.assert_allclose(vm[:, ::-1], v, atol=1e-12)
    np.testing.assert_allclose(Tm[:, ::-1], T, rtol=1e-12)


def test_bgk_limit(orc):
    """With every s equal the collision is -s (f - M^-1 fhat^eq) (the MRT
    equation reduces to lattice BGK when S = I/tau)."""
    w = W.random_smooth(10, 8, seed=11, amp=0.1)
    s0 = 0.3 / w.dt
    g = _grid(orc, w, s=np.full(16, s0))
    f = g.f + 1e-3 * np.random.default_rng(0).standard_normal(g.f.shape)
    f1 = orc.step(g, f)
    g0 = _grid(orc, w, s=np.zeros(16))
    adv = orc.step(g0, f)          # S = 0: advection only
    r, u, v, T = orc.macro(g, f)
    feq = np.stack([orc.feq(r[y, x], u[y, x], v[y, x], T[y, x], w.b)
                    for y in range(w.ny) for x in range(w.nx)], axis=1).reshape(16, w.ny, w.nx)
    want = adv - w.dt * s0 * (f - feq)
    np.testing.assert_allclose(f1, want, rtol=0, atol=1e-13 * np.max(np.abs(f)))


def test_lax_wendroff_amplification(orc):
    """S = 0 decouples the 16 planes; a Fourier mode exp(i(kx x + ky y)) in
    plane i is multiplied by 1 + sum_a [-i c_a sin th_a + c_a^2 (cos th_a - 1)],
    c_a = v_ia dt/dx, th_a = k_a dx (forward Euler + Lax-Wendroff)."""
    nx, ny = 16, 12
    w = W.uniform(nx, ny)
    g = _grid(orc, w, s=np.zeros(16))
    vx, vy, _, _, _ = orc.model()
    kx, ky = 3, 2
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    thx, thy = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    phase = thx * X + thy * Y
    lam = w.dt / w.dx
    for i in range(16):
        f = np.zeros((16, ny, nx))
        f[i] = np.cos(phase)
        out = orc.step(g, f)[i]
        cx, cy = vx[i] * lam, vy[i] * lam
        G = 1 + (-1j * cx * np.sin(thx) + cx * cx * (np.cos(thx) - 1)) \
              + (-1j * cy * np.sin(thy) + cy * cy * (np.cos(thy) - 1))
        want = np.real(G * np.exp(1j * phase))
        np.testing.assert_allclose(out, want, atol=1e-14)


def _numpy_step(orc, w, f, gx, gy):
    """Independent dense evaluation with whole-array numpy operations."""
    vx, vy, _, M, Mi = orc.model()
    b = w.b
    fh = np.einsum("ki,iyx->kyx", M, f)
    rho, jx, jy, e = fh[0], fh[1], fh[2], fh[3]
    j2 = jx ** 2 + jy ** 2
    P = (e - j2 / rho) / b
    T = P / rho
    dj = jx ** 2 - jy ** 2
    fe = np.stack([rho, jx, jy, e, 2 * P + j2 / rho, dj / rho, jx * jy / rho,
                   (e + 2 * P) * jx / rho, (e + 2 * P) * jy / rho,
                   (4 * P + j2 / rho) * jx / rho, (4 * P + j2 / rho) * jy / rho,
                   (2 * P + dj / rho) * jx / rho, (-2 * P + dj / rho) * jy / rho,
                   2 * (b + 2) * rho * T ** 2 + (6 + b) * T * j2 / rho + j2 ** 2 / rho ** 3,
                   ((b + 4) * P + j2 / rho) * jx * jy / rho ** 2,
                   ((b + 4) * P + j2 / rho) * dj / rho ** 2])
    om = -np.einsum("ik,kyx->iyx", Mi, w.s[:, None, None] * (fh - fe))
    # padded array with ghosts: x fixed (gx), y periodic
    pad = np.zeros((16, w.ny + 2, w.nx + 2))
    pad[:, 1:-1, 1:-1] = f
    pad[:, 1:-1, 0] = gx[:, 0, :]
    pad[:, 1:-1, -1] = gx[:, 1, :]
    pad[:, 0, 1:-1] = f[:, -1, :]
    pad[:, -1, 1:-1] = f[:, 0, :]
    c = pad[:, 1:-1, 1:-1]
    xp, xm = pad[:, 1:-1, 2:], pad[:, 1:-1, :-2]
    yp, ym = pad[:, 2:, 1:-1], pad[:, :-2, 1:-1]
    lam = w.dt / w.dx
    cx = (vx * lam)[:, None, None]
    cy = (vy * lam)[:, None, None]
    adv = (-0.5 * cx * (xp - xm) + 0.5 * cx ** 2 * (xp - 2 * c + xm)
           - 0.5 * cy * (yp - ym) + 0.5 * cy ** 2 * (yp - 2 * c + ym))
    return f + adv + w.dt * om


def test_dense_numpy_step_agrees(orc):
    w = W.random_smooth(7, 5, seed=5, amp=0.2, bc_x=W.BC_FIXED_EQ)
    g = _grid(orc, w)
    f = g.f.copy()
    for _ in range(5):
        want = _numpy_step(orc, w, f, g.gx, g.gy)
        got = orc.step(g, f)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.max(np.abs(want)))
        f = got
