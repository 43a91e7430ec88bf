"""Pins of the reflecting wall (Sect. (d)): a wall at the low x end whose
ghost holds the adjacent cell's distributions with every velocity mirrored
across the wall.  Because the step is covariant under x-mirroring (pinned
in test_oracle_step), a run on nx cells with that wall must equal the right
half of a run on 2 nx cells whose left half is the mirror image of the
initial state: that doubled domain stays symmetric about its centre face,
so the centre face acts as the wall.  Both runs use fixed-equilibrium ends
elsewhere; the mirror image is built here from the velocity table alone."""
import numpy as np
import pytest

import oracle
from paper_1004_5442_gb300 import workloads as W


def _mirror_perm(vx, vy):
    return [int(np.argmin(np.hypot(vx + vx[i], vy - vy[i]))) for i in range(16)]


@pytest.mark.parametrize("bc_y", [oracle.BC_PERIODIC, oracle.BC_FIXED_EQ])
def test_wall_equals_mirrored_doubled_domain(orc, bc_y):
    nx, ny, nsteps = 24, 7, 60
    w = W.random_smooth(nx, ny, seed=13, amp=0.15, nsteps=nsteps)
    vx, vy, _, _, _ = orc.model()
    perm = _mirror_perm(vx, vy)
    assert sorted(perm) == list(range(16)) and perm != list(range(16))
    g = orc.create(nx, ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, orc.BC_REFLECT_FIXED, bc_y)
    orc.run(g, nsteps)
    # doubled domain: mirror image on the left (u_x reversed), original on the right
    mirror = lambda a: a[:, ::-1]
    rho2 = np.hstack([mirror(w.rho), w.rho])
    ux2 = np.hstack([-mirror(w.ux), w.ux])
    uy2 = np.hstack([mirror(w.uy), w.uy])
    T2 = np.hstack([mirror(w.T), w.T])
    d = orc.create(2 * nx, ny, w.dx, w.dt, w.b, w.s, rho2, ux2, uy2, T2, orc.BC_FIXED_EQ, bc_y)
    orc.run(d, nsteps)
    scale = np.max(np.abs(g.f))
    np.testing.assert_allclose(g.f, d.f[:, :, nx:], rtol=0, atol=1e-13 * scale)
    # and the doubled run really is mirror-symmetric (the left half is the
    # mirror image of the right with mirrored velocities)
    np.testing.assert_allclose(d.f[perm][:, :, :nx][:, :, ::-1], d.f[:, :, nx:], rtol=0, atol=1e-13 * scale)


def test_wall_is_impermeable(orc):
    """No mass crosses the wall: with a fixed inflow state equal to a gas at
    rest, the x momentum flux through the wall is pressure only, so the total
    mass changes only by what the high end lets in (zero at rest)."""
    nx, ny = 40, 4
    w = W.random_smooth(nx, ny, seed=3, amp=0.1, nsteps=0)
    rho = w.rho.copy()
    ux = w.ux.copy()
    rho[:, -10:] = 1.0      # a gas at rest next to the high end; a step
    ux[:, -10:] = 0.0       # carries disturbances one cell, so 5 steps stay clear of it
    g = orc.create(nx, ny, w.dx, w.dt, w.b, w.s, rho, ux, 0 * ux, np.ones_like(rho), orc.BC_REFLECT_FIXED,
                   orc.BC_PERIODIC)
    m0 = orc.totals(g)[0]
    orc.run(g, 5)      # disturbances have not reached the high end yet
    assert abs(orc.totals(g)[0] - m0) <= 1e-13 * m0
