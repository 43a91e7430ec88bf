"""Pins of the oracle's ADV_LWFULL reading of the time scheme: the
Lax-Wendroff (second-order Taylor) step of the whole kinetic equation,
Eq. 3 with its collision term, f^{n+1} = f + dt f_t + (dt^2/2) f_tt.

* With every rate zero it is the unsplit Lax-Wendroff operator, bit for bit.
* On a uniform state a non-conserved moment k displaced by eps from its
  equilibrium relaxes in one step by 1 - sigma_k + sigma_k^2/2 (the
  second-order Taylor polynomial of exp(-sigma_k): on a uniform state the
  conserved moments, hence the equilibria, stay fixed, so the collision is
  linear there), where the method's forward-Euler reading gives 1 - sigma_k.
* It conserves mass, momentum and energy on a periodic grid, and commutes
  with the x mirror.
* Linearised about quadrant 3 of the four-quadrant problem and about the
  left state of the gamma = 5/3 colliding shocks it still has spectral
  radius > 1 (the Fourier-mode matrices of tests/test_oracle_stability.py):
  carrying the collision term through the second-order step does not remove
  the growth of disturbances that makes those problems lose positivity.
"""
import importlib.util
import os

import numpy as np
import pytest

from paper_1004_5442_gb300 import workloads as W


def _grid(orc, w, adv, s=None):
    return orc.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s if s is None else s, w.rho, w.ux, w.uy, w.T,
                      w.bc_x, w.bc_y, advection=adv)


@pytest.mark.parametrize("bcx,bcy", [(0, 0), (1, 0), (2, 1)])
def test_zero_rates_give_the_unsplit_operator(orc, bcx, bcy):
    w = W.random_smooth(23, 17, seed=4, amp=0.1, bc_x=bcx, bc_y=bcy)
    zero = np.zeros(16)
    a = orc.step(_grid(orc, w, orc.ADV_LWFULL, zero))
    b = orc.step(_grid(orc, w, orc.ADV_LW2D, zero))
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("k", [4, 5, 6, 7, 9, 12, 13, 15])
def test_uniform_relaxation_is_second_order_taylor(orc, k):
    sigma = np.array([0.3, 0.45, 0.6, 0.75, 0.9, 1.05, 1.2, 1.35, 1.5, 1.65, 1.8, 1.95, 0.5, 0.8, 1.1, 1.4])
    w = W.uniform(5, 4, rho=1.2, ux=0.3, uy=-0.2, T=0.9)
    s = sigma / w.dt
    _, _, _, M, Minv = orc.model()
    eps = 1e-3
    for adv, factor in ((orc.ADV_LWFULL, 1 - sigma[k] + sigma[k] ** 2 / 2), (orc.ADV_LW, 1 - sigma[k])):
        g = _grid(orc, w, adv, s)
        meq = np.tensordot(M, g.f, 1)
        f = g.f + eps * Minv[:, k][:, None, None]
        m1 = np.tensordot(M, orc.step(g, f), 1) - meq
        want = np.zeros(16)
        want[k] = eps * factor
        assert np.max(np.abs(m1 - want[:, None, None])) <= 1e-12, (adv, k)


def test_conservation_and_mirror(orc):
    w = W.random_smooth(31, 19, seed=9, amp=0.1)
    g = _grid(orc, w, orc.ADV_LWFULL)
    f1 = orc.step(g)
    _, _, _, M, _ = orc.model()
    for k in range(4):
        m0, m1 = np.tensordot(M[k], g.f, 1), np.tensordot(M[k], f1, 1)
        assert abs(m1.sum() - m0.sum()) <= 1e-13 * np.abs(m0).sum(), k
    # x mirror: reverse x and swap each velocity with its x mirror image
    vx, vy, e2, _, _ = orc.model()
    mirror = [next(j for j in range(16) if abs(vx[j] + vx[i]) < 1e-12 and abs(vy[j] - vy[i]) < 1e-12
                   and e2[j] == e2[i]) for i in range(16)]
    fm = g.f[mirror][:, :, ::-1].copy()
    np.testing.assert_allclose(orc.step(g, fm), f1[mirror][:, :, ::-1], rtol=0, atol=1e-14 * np.max(np.abs(f1)))


def _stability():
    path = os.path.join(os.path.dirname(__file__), "test_oracle_stability.py")
    spec = importlib.util.spec_from_file_location("stability_pins", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_growth_at_the_unstable_states_remains(orc):
    st = _stability()
    sig4 = st._sigma(0.03, 0.2, 0.03)
    q3 = (0.138, 1.206, 1.206, 0.029 / 0.138)
    sig2 = np.full(16, 0.1)
    sig2[4], sig2[5] = 0.005, 0.01
    left = (5.99924, 19.5975, 0.0, 76.8254)
    for state, gamma, sig, dtdx in ((q3, 1.4, sig4, 0.005), (left, 5 / 3, sig2, 1e-6 / 0.002)):
        r_full = st._radius(orc, state, gamma, sig, dtdx, advection=orc.ADV_LWFULL)
        r_euler = st._radius(orc, state, gamma, sig, dtdx)
        assert r_full > 1.0 + 1e-4, (state, r_full)
        assert r_euler > 1.0 + 1e-4, (state, r_euler)
        assert abs(r_full - r_euler) < 0.2 * (r_euler - 1.0), (state, r_full, r_euler)


def test_kinetic_equation_itself_grows_at_the_unstable_states(orc):
    """Eq. 3 linearised about a uniform equilibrium, exact in space and time:
    a Fourier mode exp(i k.x) evolves by d/dt = -i k.v + J, with J =
    -Minv S (I - JE) M the collision Jacobian (JE = d fhat^eq / d fhat, the
    oracle's complex-step Jacobian in its first four columns).  At the
    four-quadrant problem's quadrants 2 and 3 it has eigenvalues with
    positive real part at resolved wavenumbers (k dx <= 1, at the paper's
    dt = 0.005 dx, rates per dt), where quadrant 1 has none: the growth is a
    property of the kinetic equation at those states, which no consistent
    time scheme removes.  Their equilibria also have negative members."""
    vx, vy, _, M, Minv = orc.model()
    gamma = 1.4
    b = 2.0 / (gamma - 1.0)
    sig = np.full(16, 0.03)
    sig[7] = sig[8] = 0.2
    dx_over_dt = 200.0

    def max_growth(state):
        rho, ux, uy, T = state
        J4 = orc.feq_jacobian(rho, rho * ux, rho * uy, b * rho * T + rho * (ux * ux + uy * uy), b)
        JE = np.zeros((16, 16))
        JE[:, :4] = J4
        L = -Minv @ np.diag(sig) @ (np.eye(16) - JE) @ M
        worst = -np.inf
        for kdx in (0.4, 0.8, 1.0):
            k = kdx / dx_over_dt
            for ang in np.linspace(0, 2 * np.pi, 49):
                A = -1j * k * (np.cos(ang) * np.diag(vx) + np.sin(ang) * np.diag(vy)) + L
                worst = max(worst, float(np.max(np.linalg.eigvals(A).real)))
        return worst

    q1 = (1.5, 0.0, 0.0, 1.0)
    q2 = (0.5323, 1.206, 0.0, 0.3 / 0.5323)
    q3 = (0.138, 1.206, 1.206, 0.029 / 0.138)
    assert max_growth(q1) <= 1e-12
    assert max_growth(q2) > 1e-6
    assert max_growth(q3) > 1e-4
    for state in (q2, q3):
        assert np.min(orc.feq(*state, b)) < 0
