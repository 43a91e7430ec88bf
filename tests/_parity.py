"""Shared helpers for the GPU-vs-oracle parity tests."""
import numpy as np

import oracle
from paper_1004_5442_gb300 import binding as Bd


def run_oracle(w, nsteps=None):
    g = oracle.create(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy, w.T, w.bc_x, w.bc_y)
    oracle.run(g, w.nsteps if nsteps is None else nsteps)
    return g


def run_gpu(w, precision, kernel=Bd.KERNEL_AUTO, nsteps=None, tile=0):
    grid = Bd.Grid.from_workload(w, precision=precision, kernel=kernel, tile=tile)
    grid.step(w.nsteps if nsteps is None else nsteps)
    return grid


def field_errors(got, want):
    """L-inf and L1 errors of (rho, ux, uy, T), each relative to its field's
    scale; the two velocity components share the flow-speed scale."""
    names = ("rho", "ux", "uy", "T")
    U = max(np.max(np.abs(want[1])), np.max(np.abs(want[2])), 1e-12)
    Ul1 = np.mean(np.hypot(want[1], want[2])) + 1e-300
    out = {}
    for name, a, b in zip(names, got, want):
        d = np.abs(a - b)
        if name in ("ux", "uy"):
            out[name] = (np.max(d) / U, np.mean(d) / max(Ul1, 1e-12 * U))
        else:
            out[name] = (np.max(d) / np.max(np.abs(b)), np.mean(d) / np.mean(np.abs(b)))
    return out


def assert_parity(got, want, linf=None, l1=None, label=""):
    errs = field_errors(got, want)
    for name, (ei, e1) in errs.items():
        if linf is not None:
            assert ei <= linf, f"{label} {name}: Linf {ei:.3e} > {linf:.1e} ({errs})"
        if l1 is not None:
            assert e1 <= l1, f"{label} {name}: L1 {e1:.3e} > {l1:.1e} ({errs})"
    return errs


def oracle_macro_job(w, nsteps, threads):
    """(rho, ux, uy, T) of an oracle run of workload w after nsteps steps,
    with `threads` OpenMP threads; the job of one worker process."""
    oracle.set_threads(int(threads))
    return oracle.macro(run_oracle(w, nsteps))


def oracle_totals_job(w, nsteps, threads):
    """(macro fields, totals) of an oracle run of w after nsteps steps."""
    oracle.set_threads(int(threads))
    g = run_oracle(w, nsteps)
    return oracle.macro(g), oracle.totals(g)


def _cone(a, y0, x0, size, r):
    n0, n1 = a.shape
    ys = np.arange(y0 - r, y0 + size + r) % n0
    xs = np.arange(x0 - r, x0 + size + r) % n1
    return np.ascontiguousarray(a[np.ix_(ys, xs)])


def oracle_window_job(w, y0, x0, size, r):
    """(rho, ux, uy, T) on the size x size window at (y0, x0) of a periodic
    workload after r oracle steps, from a run on the window's dependency
    cone (the window widened by r cells on every side, wrapped, periodic on
    the cone itself): with a radius-1 stencil the cone's wrong edges spoil
    only the r - 1 cells next to them by step r."""
    oracle.set_threads(1)
    fields = [_cone(a, y0, x0, size, r) for a in (w.rho, w.ux, w.uy, w.T)]
    m = size + 2 * r
    g = oracle.create(m, m, w.dx, w.dt, w.b, w.s, *fields)
    oracle.run(g, r)
    return tuple(np.ascontiguousarray(q[r:r + size, r:r + size]) for q in oracle.macro(g))


def spawn_pool(workers):
    """Process pool for oracle jobs.  Workers are started with spawn, never
    forked from a process that has touched the GPU."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    return ProcessPoolExecutor(max_workers=int(workers), mp_context=mp.get_context("spawn"))
