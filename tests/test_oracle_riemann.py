"""Pins of the exact Riemann solution (printed states and textbook values)
and of the oracle's shock-tube runs against it."""
import json
import os

import numpy as np
import pytest

from oracle import riemann
from paper_1004_5442_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def test_sod_star_state_textbook():
    d = _load("textbook_riemann.json")["sod"]
    st = riemann.star_state(d["left"], d["right"], d["gamma"])
    assert abs(st.p - d["p_star"]) < d["abs_tol"]
    assert abs(st.u - d["u_star"]) < d["abs_tol"]


def test_rankine_hugoniot_reproduces_printed_rm_state():
    """Sect. (d): a Mach 2.5 shock into (1, 0, 0, 1) at gamma 1.4 gives the
    printed right state (3.33333, -2.07063, 0, 7.125)."""
    d = _load("paper_printed_states.json")["richtmyer_meshkov"]
    rho, u, p = riemann.post_shock_state(d["mach"], d["gamma"])
    want = d["post_shock_r"]
    assert abs(rho - want["rho"]) < d["abs_tol"]
    assert abs(u - want["u"]) < d["abs_tol"]
    assert abs(p - want["p"]) < d["abs_tol"]


def test_two_d_riemann_mach_numbers_fix_gamma():
    d = _load("paper_printed_states.json")["two_d_riemann"]
    q = d["quadrants"]
    g = 1.4

    def mach(s):
        return np.hypot(s["u"], s["v"]) / np.sqrt(g * s["p"] / s["rho"])

    assert abs(mach(q["2"]) / d["mach_2_4"] - 1) < d["rel_tol"]
    assert abs(mach(q["4"]) / d["mach_2_4"] - 1) < d["rel_tol"]
    assert abs(mach(q["3"]) / d["mach_3"] - 1) < d["rel_tol"]


def test_exact_solution_conserves_flux():
    """The sampled exact solution conserves mass/momentum/energy between the
    two undisturbed states (integral form of the Euler equations)."""
    L, R, g = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4
    t = 0.2
    x = np.linspace(-1, 1, 200001)
    rho, u, p = riemann.sample(L, R, g, x / t)
    dx = x[1] - x[0]
    E = p / (g - 1) + 0.5 * rho * u * u
    mass = np.trapezoid(rho, dx=dx)
    mom = np.trapezoid(rho * u, dx=dx)
    ene = np.trapezoid(E, dx=dx)
    EL, ER = L[2] / (g - 1), R[2] / (g - 1)
    assert abs(mass - (L[0] + R[0])) < 1e-4
    assert abs(mom - t * (L[2] - R[2])) < 1e-4
    assert abs(ene - (EL + ER)) < 1e-4


def _run_tube(orc, w):
    g = orc.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    orc.run(g, w.nsteps)
    return orc.macro(g)


@pytest.mark.parametrize("kind", ["sod", "strong"])
def test_oracle_shock_position_matches_exact(orc, kind):
    if kind == "sod":
        w = W.sod_tube()                                   # 400 x 4, 2000 steps
    else:
        w = W.strong_shock(nx=512, ny=4, nsteps=2500)      # same t_end as 2048 x 8, 1e4 steps
    rho, u, v, T = _run_tube(orc, w)
    L, R = w.extra["left"], w.extra["right"]
    t = w.nsteps * w.dt
    st = riemann.star_state(L, R, w.gamma)
    x = (np.arange(w.nx) + 0.5) * w.dx
    xs_exact = 0.5 + st.shock_r * t
    xs = riemann.shock_position(x, rho[0], st.rho_r, R[0])
    assert abs(xs - xs_exact) < 2 * w.dx, (xs, xs_exact)
    # the solution is y-uniform and finite; L1 error vs exact is modest
    assert np.all(np.isfinite(rho)) and np.max(np.abs(rho - rho[:1])) < 1e-12
    ex, _, _ = riemann.sample(L, R, w.gamma, (x - 0.5) / t)
    l1 = np.mean(np.abs(rho[0] - ex)) / np.mean(np.abs(ex))
    assert l1 < 0.05, l1
