"""GPU against the FP64 oracle at the benchmark configurations themselves.

* Kelvin-Helmholtz shear layer, 1024 x 1024, 5000 FP32 steps (the 4096^2
  configuration's physics at a size the oracle finishes in minutes), on the
  default kernel and on the work-queue tile the benchmark times: rho, u, v,
  T within 1e-5 (L-inf and L1, relative to each field's scale), totals
  within 1e-5 of sum |q|.
* The 4096^2 configuration itself in the launch configuration the benchmark
  times, 50 FP32 steps from the initial state: 16 seeded 64 x 64 windows
  (periodic corners among them), each against an oracle run of 50 steps on
  its dependency cone, the window widened by 50 cells on every side (the
  stencil has radius 1, so after 50 steps nothing outside the cone reaches
  the window; the cone's own edges, wrong after the first step, spoil at
  most 49 cells inward).
* The screened 256-instance Riemann sweep, 1000 FP32 steps in one batch:
  every ny = 4 instance and 16 seeded ny = 256 instances against oracle
  runs of the same instances: L1 <= 1e-4 across the shocks; the conserved
  totals of all 256 instances within 1e-5 of the oracle's (mass and energy
  relative to their sums of |q|, momentum to the larger of sum |rho u| and
  sqrt(sum rho * sum |e|)), stored by tests/golden/write_sweep_totals.py
  (the whole sweep takes the oracle about 100 minutes of 8 cores).
* The 512^2 smooth-vortex reverse mode (500 steps, checkpoints every 50)
  against the oracle's reverse mode and its central differences, stored by
  tests/golden/write_vortex_adjoint.py (the serial oracle reverse sweep
  takes minutes): FP64 within 1e-10, FP32 within 1e-3 with the same
  upstream gradient and 5e-3 end to end.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W
from _parity import assert_parity, oracle_macro_job, oracle_totals_job, oracle_window_job, run_gpu, spawn_pool

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    oracle.lib()
    yield


def _cores():
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def test_kelvin_helmholtz_1024_5000_steps():
    w = W.kelvin_helmholtz(n=1024, nsteps=5000)
    # oracle in a spawned worker (all cores) while the GPU runs here
    with spawn_pool(1) as pool:
        fut = pool.submit(oracle_totals_job, w, w.nsteps, _cores())
        got = {}
        for tile in (0, 6):
            with run_gpu(w, Bd.FP32, kernel=Bd.KERNEL_TMA, tile=tile) as g:
                assert g.health() == Bd.MRT_OK
                got[tile] = (g.macro(), g.totals(), g.info()["tile"])
        want, tot_want = fut.result()
    # sum |q| dx^2 of rho, j_x, j_y and e, the scale of each total
    rho, ux, uy, T = want
    e = w.b * rho * T + rho * (ux * ux + uy * uy)
    scale = np.array([np.sum(np.abs(q)) for q in (rho, rho * ux, rho * uy, e)]) * w.dx * w.dx
    tiles = set()
    for tile, (macro, tot, used) in got.items():
        tiles.add(used)
        errs = assert_parity(macro, want, linf=1e-5, l1=1e-5, label=f"KH 1024^2 tile {used}")
        print(f"tile {used}:", {k: ("%.2e" % a, "%.2e" % b) for k, (a, b) in errs.items()})
        assert np.all(np.abs(tot - tot_want) <= 1e-5 * scale), (tile, tot, tot_want)
    assert 6 in tiles


def test_kelvin_helmholtz_4096_windows_after_50_steps():
    import torch
    n, size, r = 4096, 64, 50
    w = W.kelvin_helmholtz(n=n, nsteps=r, seed=0)   # the benchmark's workload (rank 0)
    rng = np.random.default_rng(404)
    corners = [(0, 0), (n - size // 2, n - size // 2), (n // 4 - size // 2, 100), (3 * n // 4 - size // 2, n - 20)]
    corners += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(12)]
    with spawn_pool(min(len(corners), _cores())) as pool:
        futs = [pool.submit(oracle_window_job, w, y0, x0, size, r) for y0, x0 in corners]
        with Bd.Grid.from_workload(w, precision=Bd.FP32, kernel=Bd.KERNEL_TMA) as g:
            assert g.info()["tile"] == 6
            g.step(r)
            assert g.health() == Bd.MRT_OK
            dev = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(4)]
            g.macro(dev)
            torch.cuda.synchronize()
            wins = []
            for y0, x0 in corners:
                ys = torch.arange(y0, y0 + size, device="cuda") % n
                xs = torch.arange(x0, x0 + size, device="cuda") % n
                wins.append(tuple(q[ys][:, xs].cpu().numpy() for q in dev))
            del dev
        worst = {}
        for (y0, x0), got, fut in zip(corners, wins, futs):
            errs = assert_parity(got, fut.result(), linf=1e-5, l1=1e-5, label=f"window ({y0}, {x0})")
            for k, (ei, e1) in errs.items():
                a, b = worst.get(k, (0.0, 0.0))
                worst[k] = (max(a, ei), max(b, e1))
    print("4096^2 windows, worst (Linf, L1):", {k: ("%.2e" % a, "%.2e" % b) for k, (a, b) in worst.items()})


def _sweep():
    with open(os.path.join(GOLDEN, "riemann_instances_screened.json")) as fh:
        return W.riemann_instances(count=256, accepted=json.load(fh)["accepted"])


def test_riemann_sweep_instances_after_1000_steps():
    ws = _sweep()
    nsteps = 1000
    thin = [i for i, w in enumerate(ws) if w.ny == 4]
    tall = [i for i, w in enumerate(ws) if w.ny == 256]
    pick = sorted(np.random.default_rng(7).choice(tall, 16, replace=False).tolist())
    with open(os.path.join(GOLDEN, "riemann_sweep_totals.json")) as fh:
        ref = json.load(fh)
    assert ref["nsteps"] == nsteps and ref["count"] == len(ws)
    cores = _cores()
    with spawn_pool(cores) as pool:
        # the tall instances first (each on a quarter of the cores), then
        # the thin ones one core each, all while the GPU runs
        futs = {i: pool.submit(oracle_macro_job, ws[i], nsteps, max(1, cores // 4)) for i in pick}
        futs.update({i: pool.submit(oracle_macro_job, ws[i], nsteps, 1) for i in thin})
        with Bd.Batch(ws) as b:
            b.step(nsteps)
            got = {i: b.grid(i).macro() for i in futs}
            health = {i: b.grid(i).health() for i in range(len(ws))}
            totals = {i: b.grid(i).totals() for i in range(len(ws))}
        # mass and energy against their sums of |q|; the momentum components
        # against the larger of sum |rho u| and sqrt(sum rho * sum |e|), the
        # instance's mass times a thermal speed: a tube's net momentum can be
        # far smaller than what its end states feed in through the ghost
        # columns every step, whose FP32 rounding the totals carry
        tot_err = {}
        for i in range(len(ws)):
            assert health[i] == Bd.MRT_OK, i
            want, sc = np.array(ref["totals"][str(i)]), np.array(ref["abs_sums"][str(i)])
            mom = max(sc[1] + sc[2], np.sqrt(sc[0] * sc[3]))
            tot_err[i] = np.max(np.abs(totals[i] - want) / np.array([sc[0], mom, mom, sc[3]]))
        worst_tot = max(tot_err.values())
        bad = {i: e for i, e in tot_err.items() if e > 1e-5}
        assert not bad, ("totals", bad)
        worst = {}
        for i in sorted(futs):
            want = futs[i].result()
            assert health[i] == Bd.MRT_OK, i
            errs = assert_parity(got[i], want, l1=1e-4, label=f"instance {i} ({ws[i].nx}x{ws[i].ny})")
            worst[i] = max(e1 for _, e1 in errs.values())
    print("sweep: largest L1 error %.2e over %d ny=4 instances, %.2e over the ny=256 ones %s; "
          "totals of all %d within %.2e of their scales"
          % (max(worst[i] for i in thin), len(thin), max(worst[i] for i in pick), pick, len(ws), worst_tot))
    assert len(worst) == len(thin) + 16


def _loss(target, dx):
    def lg(r):
        d = r - target
        return 0.5 * np.sum(d * d) * dx * dx, d * dx * dx
    return lg


def _grads(w, prec, lg, dL=None):
    with Bd.Grid.from_workload(w, precision=prec) as grid:
        grid.adjoint_record(w.rho, w.ux, w.uy, w.T, w.nsteps, 50)
        rhoN = grid.macro()[0]
        L, dL_own = lg(rhoN)
        out = grid.adjoint_backward(dL_own if dL is None else dL)
    return L, out, dL_own


def test_vortex_adjoint_512_against_oracle():
    with open(os.path.join(GOLDEN, "vortex_adjoint_512.json")) as fh:
        doc = json.load(fh)
    n, seed = doc["n"], doc["seed"]
    w = W.smooth_vortex(n=n, nsteps=doc["nsteps"])
    np.testing.assert_array_equal(w.s, doc["s"])
    lg = _loss(W.vortex_target(w), w.dx)
    cells = np.sort(np.random.default_rng(seed).choice(n * n, doc["nsample"], replace=False))
    dirs = lambda q, j: np.random.default_rng(seed + 10 * q + j).standard_normal((n, n))
    names = ("rho", "ux", "uy", "T")
    gs_ref = np.array(doc["g_s"])

    def compare(got, tol, label):
        errs = {}
        for q, name in enumerate(names):
            ref = doc["fields"][name]
            g = got[q]
            samples = np.array(ref["samples"])
            err = np.linalg.norm(g.ravel()[cells] - samples) / np.linalg.norm(samples)
            errs[name] = err
            assert err <= tol, (label, name, "samples", err)
            assert abs(np.linalg.norm(g) - ref["l2"]) <= tol * ref["l2"], (label, name, "l2")
            for j in range(doc["ndir"]):
                d = dirs(q, j)
                dot = float(np.sum(g * d))
                assert abs(dot - ref["dots"][j]) <= tol * ref["l2"] * np.linalg.norm(d), (label, name, j)
        gs = got[4]
        assert np.all(gs[:4] == 0)
        err = np.linalg.norm(gs - gs_ref) / np.linalg.norm(gs_ref)
        errs["rates"] = err
        print(f"vortex adjoint {label}: relative L2 errors", {k: "%.2e" % v for k, v in errs.items()})
        assert err <= tol, (label, "rates", err)

    L64, g64, dL64 = _grads(w, Bd.FP64, lg)
    # L sums squares of differences of order 1e-3 of rho; the FP64 step's
    # multiply-add form rounds the rho = 1 background by about eps_64 kappa
    # (kappa = sum |f_i| / rho, 47 here) per step: 1e-10 of L
    assert abs(L64 - doc["loss"]) <= 1e-10 * abs(doc["loss"])
    compare(g64, 1e-10, "fp64")
    # central differences of the oracle's loss (h = 1e-4)
    for q, name in enumerate(names):
        fd = doc["fields"][name]["fd_dir0"]
        dot = float(np.sum(g64[q] * dirs(q, 0)))
        assert abs(dot - fd) <= 1e-4 * abs(fd) + 1e-6 * doc["fields"][name]["sum_abs"] * doc["h"], (name, dot, fd)
    for k, fd in doc["rates_fd"].items():
        k = int(k)
        got = g64[4][k] * w.s[k]
        assert abs(got - fd) <= 1e-4 * abs(fd) + 1e-6 * np.max(np.abs(gs_ref * w.s)), (k, got, fd)
    # FP32 reverse sweep fed the FP64 run's upstream gradient, then end to
    # end: rho_N itself carries the FP32 rounding of f^0 (about 1e-7 of
    # rho) in every cell, which enters dL/drho_N = (rho_N - rho_tgt) dx^2
    _, g32s, _ = _grads(w, Bd.FP32, lg, dL=dL64)
    compare(g32s, 1e-3, "fp32, same upstream gradient")
    L32, g32, _ = _grads(w, Bd.FP32, lg)
    assert abs(L32 - doc["loss"]) <= 1e-4 * abs(doc["loss"])
    compare(g32, 5e-3, "fp32 end to end")
