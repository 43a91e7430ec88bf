"""Pins of the oracle's model: velocity set, M, M^-1 and the equilibria.

Each check compares the oracle with something other than its own formula:
linear algebra identities, the geometric meaning of the moment rows (their
behaviour under a 90-degree rotation of the velocity set), and the moments of
a continuous Maxwellian with (b-2) internal degrees of freedom evaluated by
Gauss-Hermite quadrature (Appendix equilibria; seven-moment relations).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_velocity_set_speeds(orc):
    # Velocity table: speeds 1, 6, 2, 3 per group of four; eta = 5/2 on group 1.
    vx, vy, e2, _, _ = orc.model()
    speeds = np.hypot(vx, vy)
    np.testing.assert_allclose(speeds, np.repeat([1.0, 6.0, 2.0, 3.0], 4), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(e2, np.r_[np.full(4, 6.25), np.zeros(12)])
    # every group is closed under +-x and +-y reflections
    for g in range(4):
        pts = {(round(a, 12), round(b, 12)) for a, b in zip(vx[4 * g:4 * g + 4], vy[4 * g:4 * g + 4])}
        assert pts == {(-a, b) for a, b in pts} == {(a, -b) for a, b in pts}


def test_M_inverse(orc):
    _, _, _, M, Mi = orc.model()
    np.testing.assert_allclose(M @ Mi, np.eye(16), atol=1e-13)
    np.testing.assert_allclose(Mi @ M, np.eye(16), atol=1e-13)
    # independent inverse (LAPACK) agrees with the oracle's Gauss-Jordan
    np.testing.assert_allclose(Mi, np.linalg.inv(M), rtol=1e-11, atol=1e-14)
    assert np.count_nonzero(np.abs(M) > 1e-12) == 176


def test_M_rotation_covariance(orc):
    """Rotating every velocity by +90 degrees, (vx, vy) -> (-vy, vx), permutes
    the columns of M and maps each moment row to a signed row of M fixed by
    the row's monomial (Appendix): m2 -> -m3, m3 -> m2, m6 -> -m6, m7 -> -m7,
    m8 -> -m9, m9 -> m8, m10 -> -m11, m11 -> m10, m12 -> m13, m13 -> -m12,
    m15 -> -m15, m16 -> -m16, the isotropic rows unchanged."""
    vx, vy, _, M, _ = orc.model()
    rx, ry = -vy, vx
    perm = []
    for i in range(16):
        j = [k for k in range(16) if abs(vx[k] - rx[i]) < 1e-12 and abs(vy[k] - ry[i]) < 1e-12]
        assert len(j) == 1
        perm.append(j[0])
    M_rot = M[:, perm]
    # (target row, source row, sign), 1-based as in the Appendix
    rules = [(1, 1, 1), (2, 3, -1), (3, 2, 1), (4, 4, 1), (5, 5, 1), (6, 6, -1), (7, 7, -1),
             (8, 9, -1), (9, 8, 1), (10, 11, -1), (11, 10, 1), (12, 13, 1), (13, 12, -1),
             (14, 14, 1), (15, 15, -1), (16, 16, -1)]
    for t, s, sg in rules:
        np.testing.assert_allclose(M_rot[t - 1], sg * M[s - 1], atol=1e-12, err_msg=f"row {t}")


def test_M_columns_golden(orc):
    """Two columns worked out by hand from the Appendix rows:
    v = (1, 0) with eta^2 = 25/4 and v = (3/sqrt2)(1, 1) with eta = 0."""
    _, _, _, M, _ = orc.model()
    col1 = [1, 1, 0, 7.25, 1, 1, 0, 7.25, 0, 1, 0, 1, 0, 7.25, 0, 7.25]
    a = 3 / np.sqrt(2)
    col13 = [1, a, a, 9, 9, 0, 4.5, 9 * a, 9 * a, 9 * a, 9 * a, 0, 0, 81, 40.5, 0]
    np.testing.assert_allclose(M[:, 0], col1, atol=1e-14)
    np.testing.assert_allclose(M[:, 12], col13, atol=1e-12)


def _maxwell_moments(rho, ux, uy, T, b, npts=14):
    """Moments of rho/(2 pi T) exp(-|v-u|^2/(2T)) with an internal energy
    zeta^2 of mean (b-2) T, for the 16 Appendix monomials (each contains
    zeta^2 at most linearly, so only its mean enters)."""
    x, w = np.polynomial.hermite_e.hermegauss(npts)
    w = w / np.sqrt(2 * np.pi)
    VX = ux + np.sqrt(T) * x[:, None]
    VY = uy + np.sqrt(T) * x[None, :]
    W2 = w[:, None] * w[None, :]
    z2 = (b - 2.0) * T
    v2 = VX ** 2 + VY ** 2
    d = VX ** 2 - VY ** 2
    mono = [np.ones_like(VX), VX, VY, v2 + z2, v2, d, VX * VY, VX * (v2 + z2), VY * (v2 + z2),
            VX * v2, VY * v2, VX * d, VY * d, v2 * (v2 + z2), VX * VY * (v2 + z2), d * (v2 + z2)]
    return np.array([rho * np.sum(W2 * m) for m in mono])


@pytest.mark.parametrize("rho,ux,uy,T,gamma", [
    (1.0, 0.0, 0.0, 1.0, 1.4),
    (5.0, 0.3, -0.2, 20.0, 1.4),
    (0.125, 1.7, 0.9, 0.8, 5.0 / 3.0),
    (5.99924, 19.5975, 0.0, 76.8254, 1.4),
    (2.0, -0.5, 0.25, 0.4, 1.1),
])
def test_equilibrium_is_maxwellian_moments(orc, rho, ux, uy, T, gamma):
    b = orc.b_of_gamma(gamma)
    jx, jy = rho * ux, rho * uy
    e = b * rho * T + (jx * jx + jy * jy) / rho
    got = orc.feq_moments(rho, jx, jy, e, b)
    want = _maxwell_moments(rho, ux, uy, T, b)
    scale = np.abs(want) + rho * max(T, 1.0) ** 2 * 1e-3
    assert np.max(np.abs(got - want) / scale) < 1e-11


def test_discrete_equilibrium_round_trip(orc):
    _, _, _, M, _ = orc.model()
    b = orc.b_of_gamma(1.4)
    for rho, ux, uy, T in [(1, 0, 0, 1), (5, 0, 0, 20), (0.7, 0.4, -1.1, 2.5)]:
        f = orc.feq(rho, ux, uy, T, b)
        m = M @ f
        jx, jy = rho * ux, rho * uy
        e = b * rho * T + rho * (ux * ux + uy * uy)
        want = orc.feq_moments(rho, jx, jy, e, b)
        scale = np.max(np.abs(want))
        np.testing.assert_allclose(m[:4], [rho, jx, jy, e], rtol=0, atol=1e-14 * scale)
        np.testing.assert_allclose(m, want, rtol=0, atol=1e-13 * scale)


def test_gamma_b_relation(orc):
    # gamma = (b+2)/b
    for g in (1.1, 1.4, 5.0 / 3.0, 2.0):
        b = orc.b_of_gamma(g)
        assert abs((b + 2.0) / b - g) < 1e-15
