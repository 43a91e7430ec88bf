"""The stored exact Riemann profiles (tests/golden/riemann_exact_profiles.json,
written by tests/golden/write_exact_riemann.py) match a fresh evaluation of
the exact solver, and the Sod entry matches the textbook star state."""
import json
import os

import numpy as np

from oracle import riemann as R

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_stored_profiles_match_exact_solver():
    with open(os.path.join(GOLD, "riemann_exact_profiles.json")) as fh:
        doc = json.load(fh)
    for key in ("sod_400x4", "strong_shock_2048x8", "colliding_shocks_gamma1.4", "colliding_shocks_gamma1.667"):
        e = doc[key]
        x = (np.arange(e["nx"]) + 0.5) * e["dx"]
        rho = R.sample(tuple(e["left"]), tuple(e["right"]), e["gamma"], (x - e["x0"]) / e["t"])[0]
        np.testing.assert_allclose(e["rho"], rho, rtol=1e-14, atol=0)
    with open(os.path.join(GOLD, "textbook_riemann.json")) as fh:
        sod = json.load(fh)["sod"]
    star = doc["sod_400x4"]["star"]
    assert abs(star["p"] - sod["p_star"]) <= sod["abs_tol"]
    assert abs(star["u"] - sod["u_star"]) <= sod["abs_tol"]
