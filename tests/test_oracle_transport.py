"""Transport pins: the oracle's linearised step against the Chapman-Enskog
Navier-Stokes equations of the paper (Eqs. 12a-d) and its speed of sound
(Sect. (a), c_s = sqrt(gamma T)).

The step is linear and translation invariant about a uniform equilibrium, so
a Fourier mode exp(i k.x) is an invariant subspace: G(k) (16x16 complex) is
measured from the oracle by central differences, and its hydrodynamic
eigenvalues lambda = exp((-Gamma - i omega) dt) are compared with
  shear (k along x, u_y):     Gamma = nu k^2,  nu = T/s_7   (Eq. 12c, s_xy term)
  shear (k along (1,1)):      Gamma = nu k^2,  nu = T/s_6   (Eq. 12b, d term)
  entropy (isobaric):         Gamma = alpha k^2, alpha = T/s_8 (Eq. 12d heat flux,
                              kappa = rho T (b+2)/(2 s_8), c_p = (b+2)/2)
  sound:                      omega = sqrt(gamma T) k,
                              Gamma = k^2/2 [T((b-2)/(b s_5) + 1/s_6) + (gamma-1) alpha]
with R = 1.  sigma = s dt is small (<= 0.02) so the O(sigma) discretisation
corrections stay below the 1% tolerance.
"""
import numpy as np
import pytest

from oracle import riemann
from paper_1004_5442_gb300 import workloads as W


def _G(orc, nx, ny, kvec, sigma, T0=1.0, gamma=1.4, cfl=0.1):
    w = W.uniform(nx, ny, T=T0, gamma=gamma, cfl=cfl)
    s = np.asarray(sigma) / w.dt
    g = orc.create(nx, ny, w.dx, w.dt, w.b, s, w.rho, 0, 0, w.T)
    f0 = g.f.copy()
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    ph = 2 * np.pi * (kvec[0] * X / nx + kvec[1] * Y / ny)
    c, sn = np.cos(ph), np.sin(ph)
    h = 1e-6
    A = np.zeros((16, 16))
    B = np.zeros((16, 16))
    for j in range(16):
        d = np.zeros_like(f0)
        d[j] = c
        out = (orc.step(g, f0 + h * d) - orc.step(g, f0 - h * d)) / (2 * h)
        A[:, j] = 2 * np.mean(out * c, axis=(1, 2))
        B[:, j] = 2 * np.mean(out * sn, axis=(1, 2))
    k2 = (2 * np.pi) ** 2 * ((kvec[0] / (nx * w.dx)) ** 2 + (kvec[1] / (ny * w.dx)) ** 2)
    return A - 1j * B, w, s, k2


def _modes(orc, G, w):
    """Eigenvalues with their macroscopic content (rho, jx, jy, e)."""
    _, _, _, M, _ = orc.model()
    ev, V = np.linalg.eig(G)
    rate = -np.log(np.abs(ev)) / w.dt
    omega = -np.angle(ev) / w.dt
    macro = np.abs(M[:4] @ V)
    order = np.argsort(rate)
    return rate[order], omega[order], macro[:, order]


def test_shear_axis_is_s7(orc):
    sig = W.default_sigma(0.01, 1.0)
    sig[5], sig[6] = 0.02, 0.01          # s_6 != s_7 to tell them apart
    G, w, s, k2 = _G(orc, 256, 3, (1, 0), sig)
    rate, omega, mac = _modes(orc, G, w)
    # the slowest mode carrying transverse momentum only
    idx = [i for i in range(16) if mac[2, i] > 10 * max(mac[0, i], mac[1, i], mac[3, i])][0]
    nu = rate[idx] / k2
    assert abs(nu / (1.0 / s[6]) - 1) < 0.01, (nu, 1 / s[6])


def _diag_shear_ratio(orc, n, s6, s7, cfl):
    sig = W.default_sigma(0.01, 1.0)
    sig[5], sig[6] = s6, s7
    G, w, s, k2 = _G(orc, n, n, (1, 1), sig, cfl=cfl)
    rate, omega, mac = _modes(orc, G, w)
    # transverse momentum along (1,-1): |jx| = |jy|, no density or energy
    cand = [i for i in range(16) if mac[1, i] > 10 * max(mac[0, i], mac[3, i])
            and abs(omega[i]) < 1e-6 * k2]
    return (rate[cand[0]] / k2) / (1.0 / s[5])


def test_shear_diagonal_is_s6(orc):
    """The diagonal mode sees the dimension-split stencil at its least
    accurate, so the check is made on a finer grid and smaller sigma, and the
    discretisation error is required to shrink under refinement."""
    coarse = _diag_shear_ratio(orc, 128, 0.01, 0.02, 0.1)
    fine = _diag_shear_ratio(orc, 256, 0.005, 0.01, 0.05)
    assert abs(fine - 1) < 0.01, fine
    assert abs(fine - 1) < 0.5 * abs(coarse - 1), (coarse, fine)


@pytest.mark.parametrize("gamma,T0", [(1.4, 1.0), (5.0 / 3.0, 0.5), (1.4, 2.0)])
def test_entropy_and_sound(orc, gamma, T0):
    sig = W.default_sigma(0.01, 0.5)       # s_8 = 0.5 s_6: Pr = 0.5
    G, w, s, k2 = _G(orc, 512, 3, (1, 0), sig, T0=T0, gamma=gamma)
    rate, omega, mac = _modes(orc, G, w)
    b = w.b
    k = np.sqrt(k2)
    alpha = T0 / s[7]
    # entropy mode: non-oscillating, density and energy, no transverse momentum
    ent = [i for i in range(16) if abs(omega[i]) < 1e-6 * k and mac[0, i] > 10 * mac[2, i]][0]
    assert abs(rate[ent] / k2 / alpha - 1) < 0.01, (rate[ent] / k2, alpha)
    # sound modes: the two slowest oscillating modes
    snd = [i for i in range(16) if abs(omega[i]) > 0.5 * k][:2]
    cs = np.sqrt(gamma * T0)
    for i in snd:
        assert abs(abs(omega[i]) / k / cs - 1) < 0.005
        nu_l = T0 * ((b - 2) / (b * s[4]) + 1.0 / s[5])
        want = 0.5 * k2 * (nu_l + (gamma - 1) * alpha)
        assert abs(rate[i] / want - 1) < 0.02, (rate[i], want)


@pytest.mark.parametrize("T0", [0.5, 1.0, 2.0])
def test_sound_speed_tube(orc, T0):
    """Sect. (a): a plate separates gas at one temperature with p1/p2 =
    1 + 1e-10; the jump positions travel at c_s = sqrt(gamma T)."""
    gamma = 1.4
    nx, ny = 400, 3
    w = W.uniform(nx, ny, T=T0, gamma=gamma, sigma=0.02, bc_x=W.BC_FIXED_EQ)
    x = (np.arange(nx) + 0.5) / nx
    dp = 1e-10
    p = np.where(x < 0.5, 1 + dp, 1.0) * T0
    rho = np.broadcast_to(p / T0, (ny, nx)).copy()
    g = orc.create(nx, ny, w.dx, w.dt, w.b, w.s, rho, 0, 0, T0, orc.BC_FIXED_EQ, orc.BC_PERIODIC)
    cs = np.sqrt(gamma * T0)
    steps = int(0.3 / cs / w.dt)
    orc.run(g, steps)
    r, u, v, TT = orc.macro(g)
    pp = (r * TT)[1] / T0 - 1
    pos = riemann.shock_position(x, pp, dp / 2, 0.0)
    c_meas = (pos - 0.5) / (steps * w.dt)
    assert abs(c_meas / cs - 1) < 0.01, (c_meas, cs)
