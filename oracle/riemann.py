"""Exact Riemann solution of the 1-D Euler equations for an ideal gas.

TEST INFRASTRUCTURE ONLY (a pin for the oracle's shock-tube runs).  The
paper compares its 1-D Riemann runs with "exact solutions" (Sect. (b),
one-dimensional Riemann problem); this module is that exact solution,
written from the Rankine-Hugoniot jump conditions and the isentropic
rarefaction relations of a polytropic gas p = rho R T with R = 1 and
gamma = (b+2)/b.

Star pressure p* solves  F_L(p) + F_R(p) + (u_R - u_L) = 0  with
  shock (p > p_K):        F_K = (p - p_K) sqrt(A_K / (p + B_K)),
                          A_K = 2/((g+1) rho_K), B_K = (g-1)/(g+1) p_K
  rarefaction (p <= p_K): F_K = 2 c_K/(g-1) ((p/p_K)^((g-1)/(2g)) - 1)
and u* = (u_L + u_R)/2 + (F_R(p*) - F_L(p*))/2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.optimize import brentq


@dataclass
class StarState:
    p: float
    u: float
    rho_l: float       # density left of the contact
    rho_r: float       # density right of the contact
    shock_l: float | None   # speed of a left-facing shock (None if rarefaction)
    shock_r: float | None   # speed of a right-facing shock (None if rarefaction)


def _F(p, rho, pk, g):
    c = math.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(left, right, gamma: float) -> StarState:
    """left/right = (rho, u, p).  Returns the star region state."""
    rl, ul, pl = map(float, left)
    rr, ur, pr = map(float, right)
    g = gamma
    fun = lambda p: _F(p, rl, pl, g) + _F(p, rr, pr, g) + (ur - ul)
    lo, hi = 1e-14 * min(pl, pr), 10.0 * max(pl, pr)
    while fun(hi) < 0.0:
        hi *= 10.0
    p = brentq(fun, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    u = 0.5 * (ul + ur) + 0.5 * (_F(p, rr, pr, g) - _F(p, rl, pl, g))
    gm = (g - 1.0) / (g + 1.0)
    if p > pl:
        rho_l = rl * (p / pl + gm) / (gm * p / pl + 1.0)
        cl = math.sqrt(g * pl / rl)
        sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * p / pl + (g - 1.0) / (2.0 * g))
    else:
        rho_l = rl * (p / pl) ** (1.0 / g)
        sl = None
    if p > pr:
        rho_r = rr * (p / pr + gm) / (gm * p / pr + 1.0)
        cr = math.sqrt(g * pr / rr)
        sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * p / pr + (g - 1.0) / (2.0 * g))
    else:
        rho_r = rr * (p / pr) ** (1.0 / g)
        sr = None
    return StarState(p, u, rho_l, rho_r, sl, sr)


def sample(left, right, gamma: float, xi: np.ndarray):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t."""
    rl, ul, pl = map(float, left)
    rr, ur, pr = map(float, right)
    g = gamma
    st = star_state(left, right, gamma)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for n, s in np.ndenumerate(xi):
        if s <= st.u:  # left of the contact
            if st.p > pl:  # left shock
                if s <= st.shock_l:
                    v = (rl, ul, pl)
                else:
                    v = (st.rho_l, st.u, st.p)
            else:  # left rarefaction
                c_star = cl * (st.p / pl) ** ((g - 1.0) / (2.0 * g))
                head, tail = ul - cl, st.u - c_star
                if s <= head:
                    v = (rl, ul, pl)
                elif s >= tail:
                    v = (st.rho_l, st.u, st.p)
                else:
                    k = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * cl) * (ul - s)
                    v = (rl * k ** (2.0 / (g - 1.0)),
                         2.0 / (g + 1.0) * (cl + (g - 1.0) / 2.0 * ul + s),
                         pl * k ** (2.0 * g / (g - 1.0)))
        else:  # right of the contact
            if st.p > pr:
                if s >= st.shock_r:
                    v = (rr, ur, pr)
                else:
                    v = (st.rho_r, st.u, st.p)
            else:
                c_star = cr * (st.p / pr) ** ((g - 1.0) / (2.0 * g))
                head, tail = ur + cr, st.u + c_star
                if s >= head:
                    v = (rr, ur, pr)
                elif s <= tail:
                    v = (st.rho_r, st.u, st.p)
                else:
                    k = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * cr) * (ur - s)
                    v = (rr * k ** (2.0 / (g - 1.0)),
                         2.0 / (g + 1.0) * (-cr + (g - 1.0) / 2.0 * ur + s),
                         pr * k ** (2.0 * g / (g - 1.0)))
        rho[n], u[n], p[n] = v
    return rho, u, p


def post_shock_state(mach: float, gamma: float, rho0=1.0, p0=1.0, direction=-1):
    """State behind a normal shock of Mach `mach` running into gas at rest
    (rho0, 0, p0); direction -1 = shock moving towards -x.  Rankine-Hugoniot:
      p1/p0 = 1 + 2g/(g+1) (M^2 - 1),  rho1/rho0 = (g+1) M^2 / ((g-1) M^2 + 2),
      u1 = direction * M c0 (1 - rho0/rho1)."""
    g = gamma
    M2 = mach * mach
    p1 = p0 * (1.0 + 2.0 * g / (g + 1.0) * (M2 - 1.0))
    rho1 = rho0 * (g + 1.0) * M2 / ((g - 1.0) * M2 + 2.0)
    c0 = math.sqrt(g * p0 / rho0)
    u1 = direction * mach * c0 * (1.0 - rho0 / rho1)
    return rho1, u1, p1


def shock_position(x: np.ndarray, rho: np.ndarray, rho_behind: float, rho_ahead: float) -> float:
    """Right-most x where rho crosses (rho_behind + rho_ahead)/2, scanning from
    the right end, with linear interpolation between cell centres."""
    level = 0.5 * (rho_behind + rho_ahead)
    sgn = np.sign(rho - level)
    for i in range(len(x) - 1, 0, -1):
        if sgn[i] != sgn[i - 1]:
            t = (level - rho[i - 1]) / (rho[i] - rho[i - 1])
            return float(x[i - 1] + t * (x[i] - x[i - 1]))
    return float("nan")
