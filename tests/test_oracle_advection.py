"""Pins of the oracle's other space discretisations.

ADV_LW2D, the unsplit two-dimensional Lax-Wendroff operator (the method's
axis-by-axis operator plus the mixed term c_x c_y d_xy f of the second-order
Taylor expansion in time): its Fourier amplification factor, second-order
convergence in time for the diagonal velocities (the split operator is first
order there), conservation, the corners beyond two fixed ends, the wall as a
mirrored doubled domain, and the transpose of the step.

ADV_MINMOD / ADV_VANLEER, the flux-limited forms (first-order upwind flux
plus the Lax-Wendroff correction scaled by a limiter, per velocity and axis):
equality with Lax-Wendroff where every ratio of successive differences is 1,
the textbook upwind scheme on a sawtooth, the TVD bounds in pure advection,
conservation, the transpose of the step, and the finding that limiting the
16 distributions one by one loses positivity on the Sod tube."""
import numpy as np
import pytest

from paper_1004_5442_gb300 import workloads as W


def _grid(orc, w, adv, s=None):
    return orc.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s if s is None else s, w.rho, w.ux, w.uy, w.T,
                      w.bc_x, w.bc_y, advection=adv)


def _mode(nx, ny, kx, ky, amp=0.01):
    """Density mode 1 + amp cos(2 pi (kx x + ky y)) at rest, T = 1: every
    f_i is a_i + b_i cos(phase), since f^eq is linear in rho at fixed u, T."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    Y, X = np.meshgrid(y, x, indexing="ij")
    phase = 2 * np.pi * (kx * X + ky * Y)
    return W.uniform(nx, ny, rho=1.0, T=1.0, gamma=1.4), phase


@pytest.mark.parametrize("adv", ["lw", "lw2d"])
def test_fourier_amplification(orc, adv):
    """With S = 0 each f_i is advected on its own; on the mode e^{i(tx x +
    ty y)} the unsplit operator multiplies by G = 1 - i cx sin tx - i cy sin ty
    - cx^2 (1 - cos tx) - cy^2 (1 - cos ty) - cx cy sin tx sin ty, the split
    one by the same G without the last term."""
    nx, ny, kx, ky = 24, 16, 5, 3
    w, phase = _mode(nx, ny, kx, ky)
    w.rho = 1.0 + 0.01 * np.cos(phase)
    w.dt = 0.9 * w.dx / 6.0           # CFL 0.9: large c, so the mixed term is visible
    code = orc.ADV_LW2D if adv == "lw2d" else orc.ADV_LW
    g = _grid(orc, w, code, s=np.zeros(16))
    f1 = orc.step(g)
    vx, vy, _, _, _ = orc.model()
    tx, ty = 2 * np.pi * kx / nx, 2 * np.pi * ky / ny
    for i in range(16):
        a = g.f[i].mean()
        b = (g.f[i] - a).ravel() @ np.cos(phase).ravel() / (np.cos(phase).ravel() @ np.cos(phase).ravel())
        np.testing.assert_allclose(g.f[i], a + b * np.cos(phase), rtol=0, atol=1e-15)
        cx, cy = vx[i] * w.dt / w.dx, vy[i] * w.dt / w.dx
        G = (1 - 1j * cx * np.sin(tx) - 1j * cy * np.sin(ty) - cx * cx * (1 - np.cos(tx))
             - cy * cy * (1 - np.cos(ty)))
        if adv == "lw2d":
            G -= cx * cy * np.sin(tx) * np.sin(ty)
        want = a + b * np.real(G * np.exp(1j * phase))
        np.testing.assert_allclose(f1[i], want, rtol=0, atol=1e-15 * max(abs(a), 1.0))


def _translation_error(orc, adv, n, t_end=0.04):
    """Max error of the diagonal planes after pure advection (S = 0) of a
    smooth mode to t_end, against the exactly translated mode."""
    w, phase = _mode(n, n, 1, 1)
    w.rho = 1.0 + 0.01 * np.cos(phase)
    w.dt = 0.5 * w.dx / 6.0
    steps = int(round(t_end / w.dt))
    g = _grid(orc, w, adv, s=np.zeros(16))
    a = g.f.mean(axis=(1, 2))
    b = np.array([(g.f[i] - a[i]).ravel() @ np.cos(phase).ravel() for i in range(16)])
    b /= np.cos(phase).ravel() @ np.cos(phase).ravel()
    orc.run(g, steps)
    vx, vy, _, _, _ = orc.model()
    t = steps * w.dt
    err = 0.0
    for i in range(8, 16):
        exact = a[i] + b[i] * np.cos(phase - 2 * np.pi * (vx[i] + vy[i]) * t)
        err = max(err, np.max(np.abs(g.f[i] - exact)) / abs(b[i]))
    return err


def test_unsplit_operator_is_second_order_for_diagonal_velocities(orc):
    e_lw = [_translation_error(orc, orc.ADV_LW, n) for n in (32, 64)]
    e_2d = [_translation_error(orc, orc.ADV_LW2D, n) for n in (32, 64)]
    assert 1.7 < e_lw[0] / e_lw[1] < 2.4, e_lw      # first order: the mixed term is missing
    assert 3.5 < e_2d[0] / e_2d[1] < 4.5, e_2d      # second order
    assert e_2d[1] < 0.2 * e_lw[1]


@pytest.mark.parametrize("adv", ["lw2d", "minmod", "vanleer"])
def test_conservation_periodic(orc, adv):
    """The mixed term and the limited fluxes are differences that telescope
    on a periodic grid: rho, j, e stay constant to round-off."""
    code = {"lw2d": orc.ADV_LW2D, "minmod": orc.ADV_MINMOD, "vanleer": orc.ADV_VANLEER}[adv]
    w = W.random_smooth(20, 18, seed=4, amp=0.1)
    g = _grid(orc, w, code)
    _, _, _, M, _ = orc.model()
    t0 = orc.totals(g)
    scale = np.array([np.sum(np.abs(np.tensordot(M[k], g.f, 1))) * w.dx ** 2 for k in range(4)])
    for _ in range(10):
        orc.run(g, 1)
        assert np.all(np.abs(orc.totals(g) - t0) <= 1e-13 * scale)


def test_lw2d_corners_beyond_two_fixed_ends(orc):
    """Four uniform quadrants with fixed-equilibrium ghosts on all sides:
    the corner ghost beyond two fixed ends holds the corner cell's initial f,
    so each corner region, uniform and far from the quadrant interfaces,
    stays exactly at rest (any other quadrant's state read there would move
    it in the first step)."""
    w = W.four_quadrant_riemann(n=40)
    g = _grid(orc, w, orc.ADV_LW2D)
    f0 = g.f.copy()
    orc.run(g, 3)
    for ys in (slice(0, 4), slice(36, 40)):
        for xs in (slice(0, 4), slice(36, 40)):
            a, b = g.f[:, ys, xs], f0[:, ys, xs]
            assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    assert np.max(np.abs(g.f - f0)) > 1e-3      # the interfaces do move


@pytest.mark.parametrize("bc_y", [0, 1])
def test_lw2d_wall_equals_mirrored_doubled_domain(orc, bc_y):
    """A reflecting wall at the low x end equals the right half of the doubled
    domain whose left half is the mirror image, also with the mixed term
    (the cells next to the wall read the corners behind it)."""
    nx, ny, nsteps = 16, 7, 40
    w = W.random_smooth(nx, ny, seed=21, amp=0.15, nsteps=nsteps)
    g = orc.create(nx, ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, orc.BC_REFLECT_FIXED, bc_y,
                   advection=orc.ADV_LW2D)
    orc.run(g, nsteps)
    mirror = lambda a: a[:, ::-1]
    d = orc.create(2 * nx, ny, w.dx, w.dt, w.b, w.s, np.hstack([mirror(w.rho), w.rho]),
                   np.hstack([-mirror(w.ux), w.ux]), np.hstack([mirror(w.uy), w.uy]),
                   np.hstack([mirror(w.T), w.T]), orc.BC_FIXED_EQ, bc_y, advection=orc.ADV_LW2D)
    orc.run(d, nsteps)
    np.testing.assert_allclose(g.f, d.f[:, :, nx:], rtol=0, atol=1e-13 * np.max(np.abs(g.f)))


@pytest.mark.parametrize("adv", ["lw2d", "minmod", "vanleer"])
@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 1), (2, 0), (2, 1)])
def test_step_transpose_dot_product(orc, adv, bcx, bcy):
    """<J d, lam> = <d, J^T lam> with J d by central differences; at random
    states the limiters sit on no kink, so the tangent exists."""
    code = {"lw2d": orc.ADV_LW2D, "minmod": orc.ADV_MINMOD, "vanleer": orc.ADV_VANLEER}[adv]
    w = W.random_smooth(9, 8, seed=5, amp=0.1, bc_x=bcx, bc_y=bcy)
    g = _grid(orc, w, code)
    rng = np.random.default_rng(2)
    f = g.f * (1 + 0.01 * rng.standard_normal(g.f.shape))
    d = rng.standard_normal(f.shape)
    lam = rng.standard_normal(f.shape)
    h = 1e-7
    tangent = (orc.step(g, f + h * d) - orc.step(g, f - h * d)) / (2 * h)
    gxb, gyb, gs = np.zeros_like(g.gx), np.zeros_like(g.gy), np.zeros(16)
    adj = orc.step_adjoint(g, f, lam, gxb, gyb, gs)
    lhs, rhs = np.sum(lam * tangent), np.sum(adj * d)
    assert abs(lhs - rhs) <= 1e-7 * np.sum(np.abs(lam * tangent))
    if bcx in (1, 2) or bcy in (1, 2):
        # adjoint of the fixed ghosts (corners included for LW2D); van Leer's
        # curvature near small differences wants a smaller step
        h = 1e-8
        dgx, dgy = rng.standard_normal(g.gx.shape), rng.standard_normal(g.gy.shape)
        gx0, gy0 = g.gx.copy(), g.gy.copy()
        g.gx, g.gy = gx0 + h * dgx, gy0 + h * dgy
        fp = orc.step(g, f)
        g.gx, g.gy = gx0 - h * dgx, gy0 - h * dgy
        fm = orc.step(g, f)
        g.gx, g.gy = gx0, gy0
        t = np.sum(lam * (fp - fm) / (2 * h))
        # (behind a wall nothing is read from the ghost array, and nothing accumulates there)
        want = (np.sum(gxb * dgx) if bcx else 0.0) + (np.sum(gyb * dgy) if bcy else 0.0)
        assert abs(t - want) <= 5e-6 * max(abs(t), 1e-12)


@pytest.mark.parametrize("adv", ["minmod", "vanleer"])
def test_limited_equals_lax_wendroff_on_linear_profiles(orc, adv):
    """Where f_i is linear along both axes every ratio of successive
    differences is 1 and both limiters give phi(1) = 1: the step equals the
    method's Lax-Wendroff step (a separate code path) away from the ends."""
    code = {"minmod": orc.ADV_MINMOD, "vanleer": orc.ADV_VANLEER}[adv]
    nx, ny = 14, 12
    w = W.uniform(nx, ny, rho=1.0, T=1.0, gamma=1.4, bc_x=W.BC_FIXED_EQ, bc_y=W.BC_FIXED_EQ)
    x, y = np.arange(nx), np.arange(ny)
    Y, X = np.meshgrid(y, x, indexing="ij")
    w.rho = 1.0 + 0.01 * X + 0.02 * Y
    lim = _grid(orc, w, code)
    lw = _grid(orc, w, orc.ADV_LW)
    inner = (slice(None), slice(2, ny - 2), slice(2, nx - 2))
    a, b = orc.step(lim)[inner], orc.step(lw)[inner]
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * np.max(np.abs(b)))
    assert np.max(np.abs(orc.step(lim) - orc.step(lw))) > 1e-6   # the ends differ (theta != 1 there)


@pytest.mark.parametrize("adv", ["minmod", "vanleer"])
def test_limited_is_upwind_on_a_sawtooth(orc, adv):
    """On f_i(x) = a_i + b_i (-1)^x every ratio of successive differences is
    -1 and both limiters give phi = 0: with S = 0 each f_i takes the textbook
    first-order upwind step f - |c| (f - f_upwind)."""
    code = {"minmod": orc.ADV_MINMOD, "vanleer": orc.ADV_VANLEER}[adv]
    nx, ny = 12, 5
    w = W.uniform(nx, ny, rho=1.0, T=1.0, gamma=1.4)
    w.rho = 1.0 + 0.1 * (-1.0) ** np.tile(np.arange(nx), (ny, 1))
    g = _grid(orc, w, code, s=np.zeros(16))
    f1 = orc.step(g)
    vx, vy, _, _, _ = orc.model()
    for i in range(16):
        c = vx[i] * w.dt / w.dx
        up = np.roll(g.f[i], 1, axis=1) if c > 0 else np.roll(g.f[i], -1, axis=1)
        want = g.f[i] - abs(c) * (g.f[i] - up)
        np.testing.assert_allclose(f1[i], want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("adv", ["minmod", "vanleer"])
def test_limited_pure_advection_is_tvd(orc, adv):
    """With S = 0 each f_i on a Riemann step keeps within its initial bounds
    and its total variation along x never grows (Sweby's region holds both
    limiters for |c| <= 1); the Lax-Wendroff operator overshoots."""
    code = {"minmod": orc.ADV_MINMOD, "vanleer": orc.ADV_VANLEER}[adv]
    w = W.sod_tube(nx=120, ny=3)
    res = {}
    for name, k in (("lim", code), ("lw", orc.ADV_LW)):
        g = _grid(orc, w, k, s=np.zeros(16))
        lo, hi = g.f.min(axis=(1, 2)), g.f.max(axis=(1, 2))
        tv = np.abs(np.diff(g.f[:, 1, :], axis=1)).sum(axis=1)
        over = 0.0
        for _ in range(40):
            orc.run(g, 5)
            over = max(over, np.max(g.f.max(axis=(1, 2)) - hi), np.max(lo - g.f.min(axis=(1, 2))))
            tv_new = np.abs(np.diff(g.f[:, 1, :], axis=1)).sum(axis=1)
            if name == "lim":
                assert np.all(tv_new <= tv * (1 + 1e-13))
            tv = tv_new
        res[name] = over
    assert res["lim"] <= 1e-14
    assert res["lw"] > 1e-4


def test_limited_forms_lose_positivity_on_sod(orc):
    """Finding behind keeping the limited forms out of the GPU library: the
    discrete equilibria of this velocity set have negative members (the
    fastest diagonal group at every temperature of the benchmarks), so
    upwind-limiting the 16 distributions one by one is not positivity
    preserving, and the Sod tube loses positivity within 100 steps, while
    the method's Lax-Wendroff operator runs it to the end (2000 steps)."""
    w = W.sod_tube()
    fe = orc.feq(1.0, 0.0, 0.0, 1.0, w.b)
    assert np.all(fe[12:] < 0)
    for k in (orc.ADV_MINMOD, orc.ADV_VANLEER):
        g = _grid(orc, w, k)
        orc.run(g, 100)
        r, _, _, T = orc.macro(g)
        assert not (np.all(np.isfinite(T)) and r.min() > 0 and T.min() > 0)
    g = _grid(orc, w, orc.ADV_LW)
    orc.run(g, 100)
    r, _, _, T = orc.macro(g)
    assert r.min() > 0 and T.min() > 0
