"""Expected conserved totals of the screened 256-instance Riemann sweep (the
batched benchmark configuration) after 1000 steps, from the FP64 oracle.

Every instance of workloads.riemann_instances (the draws accepted by
screen_riemann_instances.py) is run as drawn for 1000 steps; the script
stores, per instance (its index in the sweep), the oracle's totals
(mass, x and y momentum, energy, each times dx^2) and the sums over cells of
|rho|, |rho u_x|, |rho u_y| and |e| times dx^2 (e = b rho T + rho |u|^2), the
scales a test measures the totals' error against.  The oracle takes about
100 minutes of 8 cores for the whole sweep, too slow for a test, so the
values go to riemann_sweep_totals.json beside this script.

Calls only oracle/ and the input generator.  Instances run in a pool of
single-threaded worker processes.  Run from the repository root:
    python tests/golden/write_sweep_totals.py
"""
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1004_5442_gb300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "riemann_sweep_totals.json")
NSTEPS = 1000


def _job(args):
    i, w = args
    oracle.set_threads(1)
    t0 = time.time()
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    oracle.run(g, NSTEPS)
    tot = oracle.totals(g)
    r, ux, uy, T = oracle.macro(g)
    a = w.dx * w.dx
    scale = [np.sum(np.abs(r)) * a, np.sum(np.abs(r * ux)) * a, np.sum(np.abs(r * uy)) * a,
             np.sum(np.abs(w.b * r * T + r * (ux * ux + uy * uy))) * a]
    return i, [float(v) for v in tot], [float(v) for v in scale], time.time() - t0


def main(workers=None):
    t0 = time.time()
    with open(os.path.join(HERE, "riemann_instances_screened.json")) as fh:
        ws = W.riemann_instances(count=256, accepted=json.load(fh)["accepted"])
    jobs = sorted(enumerate(ws), key=lambda iw: -iw[1].nx * iw[1].ny)   # largest first
    totals, scales = {}, {}
    with mp.get_context("spawn").Pool(workers or os.cpu_count()) as pool:
        for i, tot, sc, sec in pool.imap_unordered(_job, jobs, chunksize=1):
            totals[str(i)], scales[str(i)] = tot, sc
            print(json.dumps({"instance": i, "nx": ws[i].nx, "ny": ws[i].ny, "s": round(sec, 1)}), flush=True)
    doc = {"_source": "tests/golden/write_sweep_totals.py (FP64 oracle, each instance of the screened sweep "
                      "run as drawn for 1000 steps)",
           "nsteps": NSTEPS, "count": len(ws),
           "totals": {k: totals[k] for k in sorted(totals, key=int)},
           "abs_sums": {k: scales[k] for k in sorted(scales, key=int)},
           "seconds": round(time.time() - t0, 1)}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=0)
    print(json.dumps({"seconds": doc["seconds"], "count": doc["count"]}))


if __name__ == "__main__":
    main()
