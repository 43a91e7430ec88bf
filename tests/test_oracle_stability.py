"""Linear stability of the scheme on the uniform states of the workloads
(von Neumann): about a uniform equilibrium the step is linear and
translation invariant, so each Fourier mode exp(i k.x) is invariant and the
step acts on it as a 16 x 16 matrix G(k), measured from the oracle by
central differences on a 12 x 12 periodic grid (all wavevectors below the
Nyquist one; the grid only sets which k are sampled - the dimensionless
scheme depends on sigma, dt/dx and the state alone).

* The states of the shock tubes, the shear layer, the vortex and the
  Richtmyer-Meshkov run have spectral radius <= 1: small disturbances of
  them do not grow.
* Quadrants 2 and 3 of the four-quadrant Riemann problem (T = 0.56 and 0.21
  moving at Mach 1.36 and 3.14) have spectral radius > 1 under the
  forward-Euler reading of the time scheme: the scheme itself amplifies
  disturbances there, which is where that problem loses positivity.
"""
import numpy as np
import pytest

N = 12


def _sigma(s57, s89, others):
    x = np.full(16, float(others))
    x[4:7] = s57
    x[7:9] = s89
    return x


def _radius(orc, state, gamma, sigma, dtdx, advection=0):
    rho, ux, uy, T = state
    b = 2.0 / (gamma - 1.0)
    dx = 1.0 / N
    dt = dtdx * dx
    g = orc.create(N, N, dx, dt, b, np.asarray(sigma) / dt, rho, ux, uy, T, advection=advection)
    f0 = g.f.copy()
    X, Y = np.meshgrid(np.arange(N) + 0.5, np.arange(N) + 0.5)
    h = 1e-7 * np.max(np.abs(f0))
    worst = 0.0
    for kx in range(N // 2):
        for ky in range(N // 2):
            if kx == ky == 0:
                continue
            ph = 2 * np.pi * (kx * X + ky * Y) / N
            c, sn = np.cos(ph), np.sin(ph)
            A = np.zeros((16, 16))
            B = np.zeros((16, 16))
            for j in range(16):
                d = np.zeros_like(f0)
                d[j] = c
                out = (orc.step(g, f0 + h * d) - orc.step(g, f0 - h * d)) / (2 * h)
                A[:, j] = 2 * np.mean(out * c, axis=(1, 2))
                B[:, j] = 2 * np.mean(out * sn, axis=(1, 2))
            worst = max(worst, float(np.max(np.abs(np.linalg.eigvals(A - 1j * B)))))
    return worst


STABLE = {
    "sod left": ((1.0, 0.0, 0.0, 1.0), 1.4, _sigma(0.02, 0.71 * 0.02, 1), 0.1 / 6),
    "sod right": ((0.125, 0.0, 0.0, 0.8), 1.4, _sigma(0.02, 0.71 * 0.02, 1), 0.1 / 6),
    "strong shock left": ((5.0, 0.0, 0.0, 20.0), 1.4, _sigma(0.1, 0.1, 1), 0.05 / 6),
    "shear layer": ((1.0, 0.5, 0.0, 1.0), 5 / 3, _sigma(0.05, 0.025, 1), 0.1 / 6),
    "vortex stream": ((1.0, 0.8 * np.sqrt(1.4), 0.0, 1.0), 1.4, _sigma(0.05, 0.71 * 0.05, 1), 0.1 / 6),
    "RM post-shock": ((3.33333, -2.07063, 0.0, 7.125 / 3.33333), 1.4, _sigma(0.02, 1, 1), 0.01),
    "RM light gas": ((0.1358, 0.0, 0.0, 1 / 0.1358), 1.4, _sigma(0.02, 1, 1), 0.01),
}


@pytest.mark.parametrize("name", list(STABLE))
def test_workload_states_are_linearly_stable(orc, name):
    r = _radius(orc, *STABLE[name])
    assert r <= 1.0 + 1e-9, (name, r)


def test_four_quadrant_states_are_linearly_unstable(orc):
    sig = _sigma(0.03, 0.2, 0.03)
    r1 = _radius(orc, (1.5, 0.0, 0.0, 1.0), 1.4, sig, 0.005)
    r3 = _radius(orc, (0.138, 1.206, 1.206, 0.029 / 0.138), 1.4, sig, 0.005)
    assert r1 <= 1.0 + 1e-9
    assert r3 >= 1.001, r3
