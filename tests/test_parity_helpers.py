"""The helpers the full-size parity tests rely on, checked on the CPU: an
oracle run on a window's dependency cone gives the full periodic run's
values on that window bit for bit (same per-cell arithmetic, radius-1
stencil), also for windows that wrap around the periodic corner, and the
spawned worker pool returns the same results as a run in this process."""
import numpy as np

import oracle
from paper_1004_5442_gb300 import workloads as W
from _parity import oracle_macro_job, oracle_window_job, run_oracle, spawn_pool


def test_cone_windows_equal_full_run():
    w = W.kelvin_helmholtz(n=96, nsteps=9, seed=3)
    full = oracle.macro(run_oracle(w))
    size, r = 16, 9
    corners = [(0, 0), (90, 85), (40, 7)]
    with spawn_pool(2) as pool:
        futs = [pool.submit(oracle_window_job, w, y0, x0, size, r) for y0, x0 in corners]
        whole = pool.submit(oracle_macro_job, w, w.nsteps, 1)
        for (y0, x0), fut in zip(corners, futs):
            ys = np.arange(y0, y0 + size) % w.ny
            xs = np.arange(x0, x0 + size) % w.nx
            for got, want in zip(fut.result(), full):
                np.testing.assert_array_equal(got, want[np.ix_(ys, xs)])
        for got, want in zip(whole.result(), full):
            np.testing.assert_array_equal(got, want)
