"""Exact Riemann solutions for the tube configurations, written to
riemann_exact_profiles.json beside this script: density at the cell centres
at the final time, the star state and the shock positions.

Sod tube 400 x 4 (2000 steps), strong-shock tube 2048 x 8 (10000 steps) and
the colliding shocks of Sect. (b) (1300 cells, t = 0.13, gamma 7/5 and 5/3).
Calls only oracle/ (the exact solver) and the input generator.  Run from the
repository root:
    python tests/golden/write_exact_riemann.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import riemann as R  # noqa: E402
from paper_1004_5442_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "riemann_exact_profiles.json")


def entry(w):
    t = w.nsteps * w.dt
    x0 = w.extra["x0"]
    x = (np.arange(w.nx) + 0.5) * w.dx
    left = tuple(float(v) for v in w.extra["left"])
    right = tuple(float(v) for v in w.extra["right"])
    rho = R.sample(left, right, w.gamma, (x - x0) / t)[0]
    st = R.star_state(left, right, w.gamma)
    shocks = {}
    if st.shock_l is not None:
        shocks["left"] = x0 + st.shock_l * t
    if st.shock_r is not None:
        shocks["right"] = x0 + st.shock_r * t
    return {"nx": w.nx, "dx": w.dx, "x0": x0, "t": t, "gamma": w.gamma, "left": left, "right": right,
            "star": {"p": st.p, "u": st.u, "rho_l": st.rho_l, "rho_r": st.rho_r}, "shock_x": shocks,
            "rho": [float(v) for v in rho]}


def main():
    doc = {"_source": "tests/golden/write_exact_riemann.py (oracle/riemann.py exact solver)",
           "sod_400x4": entry(W.sod_tube()),
           "strong_shock_2048x8": entry(W.strong_shock()),
           "colliding_shocks_gamma1.4": entry(W.colliding_shocks(gamma=1.4)),
           "colliding_shocks_gamma1.667": entry(W.colliding_shocks(gamma=5 / 3))}
    with open(OUT, "w") as fh:
        json.dump(doc, fh)
    print({k: (v["shock_x"] if isinstance(v, dict) else v) for k, v in doc.items()})


if __name__ == "__main__":
    main()
