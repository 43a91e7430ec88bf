"""Seeded synthetic inputs shaped like the paper's test problems.

This module is shared by the GPU path's tests/benchmark and by the oracle's
tests.  It holds none of the method's arithmetic: it only lays out initial
macroscopic fields (rho, u_x, u_y, T), grid spacing, time step and relaxation
rates.  Rates are given as sigma_k = s_k dt (dimensionless); the relaxation
rates passed to either implementation are s_k = sigma_k / dt.

Conventions:
  * unit domain in x: dx = 1/nx, dy = dx, cell centres at (i+1/2) dx;
  * CFL = v_max dt / dx with v_max = 6, the fastest discrete speed;
  * default rates: sigma_5 = sigma_6 = sigma_7 = sigma, sigma_8 = sigma_9 =
    Pr * sigma (Prandtl number Pr = s_8/s_6), and sigma = 1 for the
    remaining non-conserved moments 10..16 and for the (inactive) 1..4;
  * fields are float64 arrays of shape (ny, nx), x fastest.

Workloads (sizes of the five benchmark configurations):
  sod_tube          Sod shock tube, 400x4, gamma 1.4, Pr 0.71, CFL 0.1, 2000 steps
  strong_shock      (rho,u,p) = (5,0,100) | (1,0,1), 2048x8, Pr 1, CFL 0.05, 10000 steps
  kelvin_helmholtz  periodic double shear layer, n x n, gamma 5/3, Pr 0.5, CFL 0.1
  smooth_vortex     periodic isentropic vortex in a Ma 0.8 stream, n x n
  riemann_instances seeded tube/ripple instances of uneven size and gamma/Pr
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

BC_PERIODIC = 0
BC_FIXED_EQ = 1
BC_REFLECT_FIXED = 2   # reflecting wall at the low end, fixed inflow at the high end
V_MAX = 6.0


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float
    dt: float
    gamma: float
    Pr: float
    sigma: np.ndarray            # (16,) dimensionless rates s_k dt
    bc_x: int
    bc_y: int
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    nsteps: int
    extra: dict = field(default_factory=dict)

    @property
    def b(self) -> float:
        return 2.0 / (self.gamma - 1.0)

    @property
    def s(self) -> np.ndarray:
        """Relaxation rates s_k in 1/time."""
        return self.sigma / self.dt

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def default_sigma(sigma: float, Pr: float, others: float = 1.0) -> np.ndarray:
    out = np.full(16, others, dtype=np.float64)
    out[4] = out[5] = out[6] = sigma
    out[7] = out[8] = Pr * sigma
    return out


def _dt(nx: int, cfl: float) -> float:
    return cfl * (1.0 / nx) / V_MAX


def _tube(name, nx, ny, left, right, gamma, Pr, sigma, cfl, nsteps, x0=0.5):
    """Left/right (rho, u, p) states split at x = x0; fixed-eq x ends."""
    dx = 1.0 / nx
    x = (np.arange(nx) + 0.5) * dx
    left_mask = np.broadcast_to(x < x0, (ny, nx))
    rho = np.where(left_mask, left[0], right[0]).astype(np.float64)
    ux = np.where(left_mask, left[1], right[1]).astype(np.float64)
    p = np.where(left_mask, left[2], right[2]).astype(np.float64)
    return Workload(name, nx, ny, dx, _dt(nx, cfl), gamma, Pr,
                    default_sigma(sigma, Pr), BC_FIXED_EQ, BC_PERIODIC,
                    np.ascontiguousarray(rho), np.ascontiguousarray(ux),
                    np.zeros((ny, nx)), np.ascontiguousarray(p / rho), nsteps,
                    {"left": left, "right": right, "x0": x0})


def sod_tube(nx: int = 400, ny: int = 4, nsteps: int = 2000, sigma: float = 0.02) -> Workload:
    """Sod tube: (rho,u,p) = (1,0,1) | (0.125,0,0.1), gamma 1.4, Pr 0.71, CFL 0.1."""
    return _tube("sod", nx, ny, (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, 0.71,
                 sigma, 0.1, nsteps)


def strong_shock(nx: int = 2048, ny: int = 8, nsteps: int = 10000, sigma: float = 0.1,
                 p_left: float = 100.0) -> Workload:
    """Strong-shock tube: (5,0,p_left) | (1,0,1), gamma 1.4, Pr 1, CFL 0.05."""
    return _tube("strong_shock", nx, ny, (5.0, 0.0, p_left), (1.0, 0.0, 1.0), 1.4, 1.0,
                 sigma, 0.05, nsteps)


def kelvin_helmholtz(n: int = 4096, nsteps: int = 5000, seed: int = 0, sigma: float = 0.05,
                     ny: int | None = None) -> Workload:
    """Periodic double shear layer (unit square), rho = T = 1, gamma 5/3, Pr 0.5.

    u_x = 0.5 tanh((y - 1/4)/delta) for y < 1/2, -0.5 tanh((y - 3/4)/delta)
    otherwise, delta = 0.01; u_y = sum_{m=1..8} a_m sin(2 pi m x + phi_m) with
    a_m ~ U(0, 1e-3), phi_m ~ U(0, 2 pi) from numpy default_rng(seed).
    """
    nx = n
    ny = n if ny is None else ny
    dx = 1.0 / nx
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx * (nx / ny) if ny != nx else (np.arange(ny) + 0.5) * dx
    delta = 0.01
    Y, X = np.meshgrid(y, x, indexing="ij")
    ux = np.where(Y < 0.5, 0.5 * np.tanh((Y - 0.25) / delta), -0.5 * np.tanh((Y - 0.75) / delta))
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.0, 1e-3, 8)
    phase = rng.uniform(0.0, 2 * np.pi, 8)
    uy = np.zeros_like(X)
    for m in range(8):
        uy += amp[m] * np.sin(2 * np.pi * (m + 1) * X + phase[m])
    one = np.ones((ny, nx))
    return Workload("kelvin_helmholtz", nx, ny, dx, _dt(nx, 0.1), 5.0 / 3.0, 0.5,
                    default_sigma(sigma, 0.5), BC_PERIODIC, BC_PERIODIC,
                    one.copy(), np.ascontiguousarray(ux), np.ascontiguousarray(uy),
                    one.copy(), nsteps, {"seed": seed})


def smooth_vortex(n: int = 512, nsteps: int = 500, seed: int = 5, sigma: float = 0.05,
                  gamma: float = 1.4, Pr: float = 0.71, mach: float = 0.8,
                  eps: float = 1.0, r0: float = 0.05, centre=(0.5, 0.5)) -> Workload:
    """Isentropic vortex (strength eps, radius r0) in a uniform Ma stream along x.

    Background rho = T = 1, u_inf = Ma sqrt(gamma);
    du = (eps/2pi) exp((1 - r^2/r0^2)/2) (-y', x')/r0,
    dT = -(gamma-1) eps^2/(8 gamma pi^2) exp(1 - r^2/r0^2), rho = T^(1/(gamma-1)).
    """
    nx = ny = n
    dx = 1.0 / n
    c = (np.arange(n) + 0.5) * dx
    Y, X = np.meshgrid(c, c, indexing="ij")
    xr = X - centre[0]
    yr = Y - centre[1]
    r2 = (xr * xr + yr * yr) / (r0 * r0)
    g = np.exp(0.5 * (1.0 - r2))
    u_inf = mach * np.sqrt(gamma)
    ux = u_inf - eps / (2 * np.pi) * g * yr / r0
    uy = eps / (2 * np.pi) * g * xr / r0
    T = 1.0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = T ** (1.0 / (gamma - 1.0))
    return Workload("smooth_vortex", nx, ny, dx, _dt(n, 0.1), gamma, Pr,
                    default_sigma(sigma, Pr), BC_PERIODIC, BC_PERIODIC,
                    np.ascontiguousarray(rho), np.ascontiguousarray(ux),
                    np.ascontiguousarray(uy), np.ascontiguousarray(T), nsteps,
                    {"seed": seed, "eps": eps, "r0": r0, "centre": centre})


def vortex_target(w: Workload, seed: int = 5) -> np.ndarray:
    """Seeded target density: the same vortex with a perturbed strength and
    centre, carried by the free stream over the run (x-periodic shift)."""
    rng = np.random.default_rng(seed)
    eps = w.extra["eps"] * (1.0 + 0.05 * rng.uniform(-1, 1))
    off = rng.uniform(-2, 2, 2) * w.dx
    t_end = w.nsteps * w.dt
    u_inf = 0.8 * np.sqrt(w.gamma)
    cx = (w.extra["centre"][0] + off[0] + u_inf * t_end) % 1.0
    cy = w.extra["centre"][1] + off[1]
    n = w.nx
    c = (np.arange(n) + 0.5) * w.dx
    Y, X = np.meshgrid(c, c, indexing="ij")
    xr = (X - cx + 0.5) % 1.0 - 0.5
    yr = Y - cy
    r2 = (xr * xr + yr * yr) / (w.extra["r0"] ** 2)
    T = 1.0 - (w.gamma - 1.0) * eps * eps / (8.0 * w.gamma * np.pi ** 2) * np.exp(1.0 - r2)
    return np.ascontiguousarray(T ** (1.0 / (w.gamma - 1.0)))


def four_quadrant_riemann(n: int = 500, nsteps: int = 12000) -> Workload:
    """Two-dimensional Riemann problem of Sect. (c): four uniform states in
    the quadrants of the unit square, split at x = y = 1/2 (quadrant 1 upper
    right, counted counter-clockwise):
        1: (rho, u, v, T) = (1.5, 0, 0, 1)
        2: (0.5323, 1.206, 0, 0.3/0.5323)
        3: (0.138, 1.206, 1.206, 0.029/0.138)
        4: (0.5323, 0, 1.206, 0.3/0.5323)
    gamma 1.4; dx = 1/n, dt = 0.005 dx (1e-5 at the paper's n = 500, so
    t = 0.12 after 12000 steps); s_8 = s_9 = 2e4, every other rate 3e3 at
    n = 500 (sigma = s dt = 0.2 and 0.03, kept at other n); fixed-equilibrium
    ghosts on all four sides.  Pr = s_8/s_6 follows from these rates."""
    dx = 1.0 / n
    dt = 0.005 * dx
    c = (np.arange(n) + 0.5) * dx
    Y, X = np.meshgrid(c, c, indexing="ij")
    q = np.where(X >= 0.5, np.where(Y >= 0.5, 0, 3), np.where(Y >= 0.5, 1, 2))
    states = np.array([[1.5, 0.0, 0.0, 1.0],
                       [0.5323, 1.206, 0.0, 0.3 / 0.5323],
                       [0.138, 1.206, 1.206, 0.029 / 0.138],
                       [0.5323, 0.0, 1.206, 0.3 / 0.5323]])
    f = [np.ascontiguousarray(states[q, k]) for k in range(4)]
    sigma = np.full(16, 0.03)
    sigma[7] = sigma[8] = 0.2
    return Workload("four_quadrant_riemann", n, n, dx, dt, 1.4, 0.2 / 0.03, sigma, BC_FIXED_EQ, BC_FIXED_EQ,
                    f[0], f[1], f[2], f[3], nsteps, {"t_end": nsteps * dt})


def colliding_shocks(gamma: float = 1.4, mrt: bool = True, nx: int = 1300, ny: int = 4, x0: float = 0.4,
                     nsteps: int = 130000) -> Workload:
    """One-dimensional Riemann problem of Sect. (b) on the 2-D model:
    (rho, u, v, T) = (5.99924, 19.5975, 0, 76.8254) left of x0 and
    (5.99242, -6.19633, 0, 7.69222) right of it; dx = 0.002, dt = 1e-6
    (t = 0.13 after 130000 steps); x in [0, nx dx] with fixed-equilibrium
    ends (2.6 units at nx = 1300, so that no wave of either gamma reaches an
    end by t = 0.13), y periodic.  Rates: MRT s_5 = 5e3, s_6 = 1e4, every
    other s = 1e5; SRT every s = 1e5 (tau = 1e-5)."""
    dx, dt = 0.002, 1e-6
    x = (np.arange(nx) + 0.5) * dx
    left = np.broadcast_to(x < x0, (ny, nx))
    rho = np.where(left, 5.99924, 5.99242)
    ux = np.where(left, 19.5975, -6.19633)
    T = np.where(left, 76.8254, 7.69222)
    s = np.full(16, 1e5)
    if mrt:
        s[4], s[5] = 5e3, 1e4
    return Workload("colliding_shocks_" + ("mrt" if mrt else "srt"), nx, ny, dx, dt, gamma, s[7] / s[5],
                    s * dt, BC_FIXED_EQ, BC_PERIODIC, np.ascontiguousarray(rho), np.ascontiguousarray(ux),
                    np.zeros((ny, nx)), np.ascontiguousarray(T), nsteps,
                    {"x0": x0, "left": (5.99924, 19.5975, 5.99924 * 76.8254),
                     "right": (5.99242, -6.19633, 5.99242 * 7.69222)})


def richtmyer_meshkov(nx: int = 360, ny: int = 100, nsteps: int = 10400, x_shock: float = 0.25) -> Workload:
    """Richtmyer-Meshkov configuration of Sect. (d): a 0.36 x 0.1 box on
    360 x 100 cells (dx = 0.001), light gas (rho, u, v, p) = (0.1358, 0, 0, 1)
    left of the interface x = 0.24 + 0.005 sin(pi/2 + 40 pi y), heavy gas
    (1, 0, 0, 1) between it and the Mach 2.5 shock at x_shock, post-shock
    state (3.33333, -2.07063, 0, 7.125) right of the shock; reflecting wall
    on the left, fixed inflow of the post-shock state on the right, periodic
    in y; gamma 1.4, dt = 1e-5 (t = 0.104 after 10400 steps), s_5 = 2e3 and
    every other rate 1e5 (sigma = 0.02 and 1)."""
    dx = 0.36 / nx
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    Y, X = np.meshgrid(y, x, indexing="ij")
    iface = 0.24 + 0.005 * np.sin(np.pi / 2 + 40 * np.pi * Y)
    light = X < iface
    post = X >= x_shock
    rho = np.where(light, 0.1358, np.where(post, 3.33333, 1.0))
    ux = np.where(post, -2.07063, 0.0)
    p = np.where(post, 7.125, 1.0)
    sigma = np.full(16, 1.0)
    sigma[4] = 0.02
    return Workload("richtmyer_meshkov", nx, ny, dx, 1e-5, 1.4, 1.0, sigma, BC_REFLECT_FIXED, BC_PERIODIC,
                    np.ascontiguousarray(rho), np.ascontiguousarray(ux), np.zeros((ny, nx)),
                    np.ascontiguousarray(p / rho), nsteps, {"x_shock": x_shock, "t_end": nsteps * 1e-5})


def shrink(w: Workload, nsteps: int) -> Workload:
    return replace(w, nsteps=nsteps)


def uniform(nx: int, ny: int, rho=1.0, ux=0.0, uy=0.0, T=1.0, gamma=1.4, Pr=0.71,
            sigma=0.05, cfl=0.1, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC, nsteps=1) -> Workload:
    one = np.ones((ny, nx))
    return Workload("uniform", nx, ny, 1.0 / nx, _dt(nx, cfl), gamma, Pr,
                    default_sigma(sigma, Pr), bc_x, bc_y, rho * one, ux * one, uy * one,
                    T * one, nsteps)


def random_smooth(nx: int, ny: int, seed: int = 1, amp: float = 0.05, gamma=1.4, Pr=0.71,
                  sigma=0.05, cfl=0.1, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC,
                  nsteps=1) -> Workload:
    """rho, u, T = background + a few seeded low Fourier modes (amplitude amp)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    Y, X = np.meshgrid(y, x, indexing="ij")

    def field_(base):
        out = np.full((ny, nx), base, dtype=np.float64)
        for _ in range(3):
            kx, ky = rng.integers(0, 3, 2)
            ph = rng.uniform(0, 2 * np.pi)
            out += amp * rng.uniform(-1, 1) * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
        return out

    return Workload("random_smooth", nx, ny, 1.0 / nx, _dt(nx, cfl), gamma, Pr,
                    default_sigma(sigma, Pr), bc_x, bc_y, field_(1.0), field_(0.0) * 4,
                    field_(0.0) * 4, field_(1.0), nsteps, {"seed": seed})


def riemann_candidates(seed: int = 4, nx_range=(256, 4096), ny_choices=(4, 256), sigma: float = 0.02,
                       cfl: float = 0.05, nsteps: int = 1000):
    """Endless seeded stream of tube/ripple instances of uneven size, gamma, Pr
    and pressure ratio; yields (draw index, Workload).

    Per draw: nx ~ U{nx_range}, ny from ny_choices (fair coin),
    gamma ~ U(1.1, 1.67), Pr ~ U(0.5, 2), pi = p_L/p_R log-uniform in [10, 100];
    left (rho,u,p) = (5, 0, pi), right (1, 0, 1).  ny > 4 instances get an
    interface ripple x = 0.5 + 2 dx sin(2 pi m y / L_y), m ~ U{1..4}.
    sigma = s dt of the viscous moments (0.02: nu = 50 T dt keeps the
    under-resolved shocks of this family stable at CFL 0.05)."""
    rng = np.random.default_rng(seed)
    k = 0
    while True:
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(ny_choices[int(rng.integers(0, len(ny_choices)))])
        gamma = float(rng.uniform(1.1, 1.67))
        Pr = float(rng.uniform(0.5, 2.0))
        ratio = float(np.exp(rng.uniform(np.log(10.0), np.log(100.0))))
        m = int(rng.integers(1, 5))
        dx = 1.0 / nx
        x = (np.arange(nx) + 0.5) * dx
        y = (np.arange(ny) + 0.5) * dx
        Ly = ny * dx
        Y, X = np.meshgrid(y, x, indexing="ij")
        iface = 0.5 + (2 * dx * np.sin(2 * np.pi * m * Y / Ly) if ny > 4 else 0.0)
        left = X < iface
        rho = np.where(left, 5.0, 1.0)
        p = np.where(left, ratio, 1.0)
        w = Workload(f"draw{k}", nx, ny, dx, _dt(nx, cfl), gamma, Pr,
                     default_sigma(sigma, Pr), BC_FIXED_EQ, BC_PERIODIC,
                     np.ascontiguousarray(rho), np.zeros((ny, nx)), np.zeros((ny, nx)),
                     np.ascontiguousarray(p / rho), nsteps,
                     {"ratio": ratio, "mode": m, "draw": k})
        yield k, w
        k += 1


def riemann_instances(count: int = 256, seed: int = 4, accepted=None, **kw):
    """The first `count` draws of riemann_candidates, or, given the accepted
    draw indices of a screening, the first `count` accepted draws."""
    out = []
    keep = None if accepted is None else set(int(a) for a in accepted)
    for k, w in riemann_candidates(seed=seed, **kw):
        if keep is None or k in keep:
            out.append(w)
        if len(out) == count or (keep is not None and k > max(keep)):
            break
    return out
