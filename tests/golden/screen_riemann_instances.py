"""Screen the seeded tube/ripple draws with the FP64 oracle.

Each draw of workloads.riemann_candidates (seed 4) is run as drawn (full
nx x ny grid, ripple included) for its 1000 steps; a draw is accepted when
rho and T are finite and positive in every cell after every step, the same
admissibility the library's health flag tests each step.  Draws are taken in
order until 256 are accepted; the accepted and rejected indices are written
to riemann_instances_screened.json beside this script.

Calls only oracle/ (and the input generator).  Draws are screened in a pool
of single-threaded worker processes.  Run from the repository root:
    python tests/golden/screen_riemann_instances.py
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

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "riemann_instances_screened.json")


def first_bad_step(w, nsteps=None):
    """Step index (1-based) after which some cell has rho or T non-positive or
    non-finite; None when all nsteps states are admissible."""
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    for n in range(1, (w.nsteps if nsteps is None else nsteps) + 1):
        g.f = oracle.step(g)
        r, _, _, T = oracle.macro(g)
        if not (np.all(np.isfinite(r)) and np.all(np.isfinite(T)) and r.min() > 0 and T.min() > 0):
            return n
    return None


def accept(w) -> bool:
    return first_bad_step(w) is None


def _screen(args):
    k, w = args
    oracle.set_threads(1)
    t0 = time.time()
    bad = first_bad_step(w)
    return k, bad, time.time() - t0


def main(count=256, first_batch=300, workers=None):
    t0 = time.time()
    verdict = {}
    gen = W.riemann_candidates(seed=4)
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers or os.cpu_count()) as pool:
        todo = first_batch
        while True:
            draws = [next(gen) for _ in range(todo)]
            # largest first, so the pool stays busy to the end
            draws.sort(key=lambda kw: -kw[1].nx * kw[1].ny)
            for k, bad, sec in pool.imap_unordered(_screen, draws, chunksize=1):
                verdict[k] = bad
                print(json.dumps({"draw": k, "bad_step": bad, "s": round(sec, 1)}), flush=True)
            ks = sorted(verdict)
            acc = [k for k in ks if verdict[k] is None]
            if len(acc) >= count:
                break
            todo = count - len(acc) + 16
    last = acc[count - 1]
    acc = acc[:count]
    rej = [k for k in ks if verdict[k] is not None and k < last]
    doc = {"_source": "tests/golden/screen_riemann_instances.py (FP64 oracle, full instance, "
                      "rho and T checked after each of 1000 steps)",
           "seed": 4, "count": count, "accepted": acc, "rejected": rej,
           "first_bad_step": {str(k): verdict[k] for k in rej},
           "acceptance_rate": len(acc) / (len(acc) + len(rej)), "seconds": round(time.time() - t0, 1)}
    with open(OUT, "w") as fh:
        json.dump(doc, fh, indent=0)
    print(json.dumps({k: v for k, v in doc.items() if k not in ("accepted", "rejected", "first_bad_step")}))


if __name__ == "__main__":
    main()
