#!/usr/bin/env python3
"""Throughput benchmark of the fused MRT-FDLB step (cell-updates/s).

Workload: the 4096 x 4096 periodic Kelvin-Helmholtz double shear layer
(gamma 5/3, Pr 0.5, CFL 0.1), FP32 state and arithmetic, TMA strip kernel.
A benchmark step is one time step of the whole grid (moments, relaxation,
inverse transform, Lax-Wendroff advection and Euler update of all 16.8 M
cells).  The state (2 x 1.07 GB) is larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Reported on one JSON line (rank 0): device-timed throughput, the end-to-end
rate through the C ABI with host buffers (initial fields uploaded, totals read
back every step, final fields downloaded), the roofline of the step kernel
against the measured HBM copy bandwidth, the SM clocks seen during the timed
region, and the FP64 CPU oracle timed on a bounded sample of the same
workload.  With --gpus N > 1 (torchrun) every rank advances its own replica:
the step has no exchange between GPUs (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_CELL_F32 = 128      # 16 f_i read + 16 written, 4 bytes each
BYTES_PER_CELL_F64 = 256
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["paper_1004_5442_gb300/csrc/step_kernels.cu", "paper_1004_5442_gb300/csrc/step_strip.cuh",
                  "paper_1004_5442_gb300/csrc/tma.cuh", "paper_1004_5442_gb300/csrc/model.cuh",
                  "paper_1004_5442_gb300/csrc/internal.h"]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_tma_f32_kh4096.md")
# FP64 step, per cell-update (ncu instruction counters of a plain
# step_tma<double> launch, tile 6, profiles/step_tma_f64_kh2048.md):
# FP64-pipe thread instructions and flops (DADD 86 + DMUL 28 + 2 x DFMA 118).
# Their roof is the device's FP64 multiply-add rate, measured in the same
# run by mrt_debug_fma_rate (one DFMA = 2 flops = 1 pipe instruction).
FP64_PIPE_INST_PER_CELL = 234.0
FP64_FLOPS_PER_CELL = 350.0
EXACT_PROFILES = os.path.join(ROOT, "tests", "golden", "riemann_exact_profiles.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000, help="timed steps (5000: the 4096^2 shear-layer run)")
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=4096, help="grid edge (default 4096)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-lw2d", action="store_true")
    ap.add_argument("--adjoint-n", type=int, default=0,
                    help="time the reverse mode on one n x n shear layer (8 steps, checkpoints every 4) "
                         "instead of the default cases (for profiler captures)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-problems", action="store_true", help="skip the tube / 2-D Riemann problem runs")
    ap.add_argument("--problem-steps", type=int, default=0,
                    help="run each tube / 2-D Riemann problem for at most this many steps and report timings only "
                         "(for profiler captures; 0 = the problems' full runs with their error checks)")
    ap.add_argument("--batch-steps", type=int, default=1000, help="timed steps of the 256-instance sweep")
    ap.add_argument("--batch-count", type=int, default=256, help="instances of the sweep (first n screened draws)")
    ap.add_argument("--tile", type=int, default=0, help="TMA kernel variant (0 = library default)")
    ap.add_argument("--sweep-tiles", action="store_true", help="time every TMA variant, print one line each")
    ap.add_argument("--fma-only", action="store_true",
                    help="print the device's FP64 and FP32 multiply-add throughput (mrt_debug_fma_rate) and exit")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_init(n_gpus, backend=None):
    """Rank, world size and local rank from the launcher's environment; one
    process group (NCCL on GPUs) when the world has more than one rank."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend or "nccl")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    """Maximum of x over all ranks (the slowest replica sets the time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, steps, ms_max, world):
    """Units of all replicas per second over the slowest rank's time."""
    return world * units_per_rank * steps / (ms_max * 1e-3)


def workload_config(w, world):
    return {"workload": f"kelvin_helmholtz_{w.nx}x{w.ny}_fp32", "nx": w.nx, "ny": w.ny, "gamma": w.gamma,
            "Pr": w.Pr, "cfl": 0.1, "precision": "fp32",
            "l2": "state 2 x %.2f GB > 129 MB L2, no flush" % (16 * w.nx * w.ny * 4 / 1e9),
            "parallelism": f"replicas{world}"}


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


class NvmlClocks:
    """SM clock, power and clock-event reasons read through NVML (read-only
    queries, nothing is set) every `period` seconds in a thread, plus one
    read on demand (`sample()`), so that a timed region of a few milliseconds
    still has samples.  Falls back to ClockSampler if NVML cannot be loaded."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, local, period=0.001):
        import ctypes
        import threading
        self.period = period
        self.samples = []
        self.fallback = None
        self._stop = threading.Event()
        self._thread = None
        self.nv = None
        self.h = None
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise OSError("nvmlInit")
            h = ctypes.c_void_p()
            bus = self._pci_bus_id(local)
            rc = nv.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) if bus else 1
            if rc != 0:
                rc = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(local), ctypes.byref(h))
            if rc != 0:
                raise OSError("nvml handle")
            self.nv, self.h = nv, h
            self.reason_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
            mx = ctypes.c_uint()
            self.max_mhz = float(mx.value) if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 else None
        except Exception:
            self.fallback = ClockSampler(local)

    @staticmethod
    def _pci_bus_id(local):
        try:
            import torch
            p = torch.cuda.get_device_properties(local)
            return "%08X:%02X:%02X.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        except Exception:
            return None

    def sample(self):
        import ctypes
        if self.nv is None:
            return
        mhz, mw, r = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(mhz)) != 0:
            return
        self.nv.nvmlDeviceGetPowerUsage(self.h, ctypes.byref(mw))
        self.reason_fn(self.h, ctypes.byref(r))
        self.samples.append((float(mhz.value), mw.value / 1e3, int(r.value)))

    def _run(self):
        while not self._stop.is_set():
            self.sample()
            self._stop.wait(self.period)

    def __enter__(self):
        if self.fallback is not None:
            self.fallback.__enter__()
            return self
        import threading
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *exc):
        if self.fallback is not None:
            return self.fallback.__exit__(*exc)
        self._stop.set()
        self._thread.join()

    def summary(self):
        if self.fallback is not None:
            out = self.fallback.summary()
            out["source"] = "nvidia-smi -lms 100"
            return out
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0, "source": "nvml"}
        reasons = sorted({nm for _, _, r in self.samples for bit, nm in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(m for m, _, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "sm_mhz_min": min(m for m, _, _ in self.samples),
                "power_w_max": max(p for _, p, _ in self.samples), "reasons": reasons,
                "samples": len(self.samples), "source": "nvml read-only queries every 1 ms"}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(n):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source and states them for an n x n launch."""
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    hsh = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    size = re.search(r"traffic_grid:\s*(\d+)", text)
    if not m or not hsh or hsh.group(1) != kernel_source_hash():
        return None
    if not size or int(size.group(1)) != n:
        return None
    return float(m.group(1))


# ---------------------------------------------------------------------------
def cpu_oracle_rate(w, budget_s=12.0, max_steps=None, rows=512):
    """The FP64 oracle on a band of the workload (all nx columns, `rows`
    rows, periodic), stepped until budget_s of wall time has passed."""
    import oracle
    oracle.build()
    threads = oracle.get_threads()
    band = slice(0, rows)
    g = oracle.create(w.nx, rows, w.dx, w.dt, w.b, w.s, w.rho[band], w.ux[band], w.uy[band], w.T[band],
                      oracle.BC_PERIODIC, oracle.BC_PERIODIC)
    work = np.zeros_like(g.f)
    cfg = g.cfg()
    import ctypes
    lib = oracle.lib()
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    steps = 0
    t0 = time.perf_counter()
    while True:
        lib.orc_run(ctypes.byref(cfg), p(g.f), p(g.gx), p(g.gy), 1, p(work))
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and steps >= max_steps) or (max_steps is None and el >= budget_s and steps >= 2):
            break
    rate = w.nx * rows * steps / el
    return rate, threads, f"{w.nx}x{rows} band of the workload's initial state, periodic, {steps} oracle steps, {el:.1f} s"


# ---------------------------------------------------------------------------
def run_reference(args):
    """The oracle timed on the host cores (rank 0 only; other ranks exit
    without work)."""
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return None
    from paper_1004_5442_gb300 import workloads as W
    w = W.kelvin_helmholtz(n=args.n, nsteps=0)
    import oracle
    oracle.build()
    rows = 64
    band = slice(0, rows)
    g = oracle.create(w.nx, rows, w.dx, w.dt, w.b, w.s, w.rho[band], w.ux[band], w.uy[band], w.T[band],
                      oracle.BC_PERIODIC, oracle.BC_PERIODIC)
    oracle.run(g, max(args.warmup, 0))
    t0 = time.perf_counter()
    oracle.run(g, args.steps)
    el = time.perf_counter() - t0
    rate = w.nx * rows * args.steps / el
    sample = f"{w.nx}x{rows} band of the {args.n}^2 workload, periodic, FP64 oracle, {args.steps} steps"
    line = {"impl": "reference", "metric": "cell_updates_per_s", "value": rate, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, world),
            "cpu_baseline": {"value": rate, "unit": "cell-updates/s", "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


# ---------------------------------------------------------------------------
def unsplit_operator(Bd, w, torch, stream, args, peak):
    """The same workload stepped with MRT_ADV_LW2D: FP32 (HBM bound, the
    same 128 B per cell-update) and FP64, CUDA events on the grid's stream."""
    out = {}
    cells = w.nx * w.ny
    for prec, name, k in ((Bd.FP32, "fp32", max(20, min(1000, args.steps // 5))),
                          (Bd.FP64, "fp64", max(5, min(60, args.steps // 25)))):
        if prec == Bd.FP64 and args.no_fp64:
            continue
        with torch.cuda.stream(stream):
            g = Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_TMA, stream=stream.cuda_stream,
                                      advection=Bd.ADV_LW2D)
        g.step(3)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        g.step(k)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        assert g.health() == Bd.MRT_OK
        tile = g.info()["tile"]
        g.close()
        per = ms * 1e-3 / k
        bpc = BYTES_PER_CELL_F32 if prec == Bd.FP32 else BYTES_PER_CELL_F64
        out[name] = {"value": cells / per, "unit": "cell-updates/s", "steps": k, "tile": tile,
                     "hbm_achieved_gbs": bpc * cells / per / 1e9, "hbm_frac": bpc * cells / per / 1e9 / peak}
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    from paper_1004_5442_gb300 import build as B
    B.build()
    from paper_1004_5442_gb300 import binding as Bd
    from paper_1004_5442_gb300 import workloads as W

    w = W.kelvin_helmholtz(n=args.n, nsteps=0, seed=rank)
    cells = w.nx * w.ny
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        grid = Bd.Grid.from_workload(w, precision=Bd.FP32, kernel=Bd.KERNEL_TMA, stream=stream.cuda_stream,
                                     tile=args.tile)
    info = grid.info()
    assert info["kernel"] == Bd.KERNEL_TMA
    # warm-up
    grid.step(max(args.warmup, 3))
    torch.cuda.synchronize()
    assert grid.health() == Bd.MRT_OK

    # timed region: K steps, CUDA events on the grid's stream
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with NvmlClocks(local) as clk:
        ev0.record(stream)
        grid.step(args.steps)
        ev1.record(stream)
        clk.sample()          # the steps are queued: the GPU is busy now
        torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1)
    ms = allmax(ms, world)
    tot = grid.totals()
    assert grid.health() == Bd.MRT_OK and np.all(np.isfinite(tot))
    value = whole_job_rate(cells, args.steps, ms, world)
    per_launch_s = ms * 1e-3 / args.steps
    peak, peak_kind = measured_peak_hbm()
    achieved = BYTES_PER_CELL_F32 * cells / per_launch_s / 1e9
    traffic = profiled_traffic(w.nx if w.nx == w.ny else -1)
    grid.close()

    line = {"metric": "cell_updates_per_s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(w, world),
            "kernel": {"name": "step_tma", "tile": info["tile"]},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": BYTES_PER_CELL_F32 * cells,
                         "timing": "CUDA events on the grid's stream over K steps (K - 1 replayed from two-step "
                                   "CUDA graphs, the last one also computing the totals partials, whose two-pass "
                                   "reduction the library enqueues on the grid's side stream)"},
            # K step kernels, the last one computing the totals partials, and
            # the two passes of the totals reduction (side stream)
            "gpu_launches": args.steps + 2,
            "clocks": clk.summary()}

    # FP64 state and arithmetic (FP64 ALU bound on this part), same workload
    if not args.no_fp64:
        with torch.cuda.stream(stream):
            g64 = Bd.Grid.from_workload(w, precision=Bd.FP64, kernel=Bd.KERNEL_TMA, stream=stream.cuda_stream)
        g64.step(3)
        k64 = min(150, max(5, args.steps // 10))
        torch.cuda.synchronize()
        ev0.record(stream)
        g64.step(k64)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1)
        assert g64.health() == Bd.MRT_OK
        g64.close()
        per64 = ms64 * 1e-3 / k64
        rate64 = cells / per64
        fma64, fma_ms = Bd.fma_rate(Bd.FP64)                          # flop/s, 2 per DFMA
        pipe_peak = fma64 / 2                                          # DFMA instructions / s
        line["fp64"] = {"value": rate64, "unit": "cell-updates/s", "steps": k64,
                        "hbm_achieved_gbs": BYTES_PER_CELL_F64 * cells / per64 / 1e9,
                        "hbm_frac": BYTES_PER_CELL_F64 * cells / per64 / 1e9 / peak,
                        "roofline": {"bound": "alu", "achieved": rate64 * FP64_FLOPS_PER_CELL / 1e12,
                                     "peak": fma64 / 1e12, "unit": "TFLOP/s",
                                     "frac": rate64 * FP64_FLOPS_PER_CELL / fma64,
                                     "pipe_frac": rate64 * FP64_PIPE_INST_PER_CELL / pipe_peak,
                                     "peak_source": "measured: mrt_debug_fma_rate FP64 in this run "
                                                    f"(independent DFMA chains, {fma_ms:.1f} ms launch)",
                                     "per_cell": {"fp64_pipe_inst": FP64_PIPE_INST_PER_CELL,
                                                  "flops": FP64_FLOPS_PER_CELL}}}

    # the unsplit two-dimensional Lax-Wendroff operator (mixed term on the
    # diagonal velocities), same workload and timing, FP32 and FP64
    if not args.no_lw2d:
        line["lw2d"] = unsplit_operator(Bd, w, torch, stream, args, peak)
        if not args.no_adjoint:
            line["lw2d"]["adjoint"] = adjoint_costs(
                Bd, W, torch, stream, advection=Bd.ADV_LW2D,
                cases=[("smooth_vortex_512x512_fp32", W.smooth_vortex(n=512, nsteps=500), 500, 50)])

    # adjoint / forward cost (smooth vortex 512^2, 500 FP32 steps, checkpoints
    # every 50; and the 4096^2 workload for the HBM-bound ratio)
    if not args.no_adjoint:
        cases = None
        if args.adjoint_n > 0:
            n = args.adjoint_n
            cases = [(f"kelvin_helmholtz_{n}x{n}_fp32", W.kelvin_helmholtz(n=n, nsteps=8), 8, 4)]
        line["adjoint"] = adjoint_costs(Bd, W, torch, stream, cases=cases)

    # the paper's tube and 2-D problems: throughput next to error vs exact
    if not args.no_problems:
        line["paper_problems"] = paper_problems(Bd, W, torch, stream, peak, args.problem_steps)

    # 256 independent tube/ripple instances of uneven size, one launch per step
    if not args.no_batch:
        line["batch"] = batch_sweep(Bd, W, torch, args, peak)

    # end to end through the C ABI with pinned host buffers
    if not args.no_e2e:
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (w.rho, w.ux, w.uy, w.T)]
        outs = [torch.empty((w.ny, w.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
        p = Bd.make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, w.s, w.bc_x, w.bc_y, Bd.FP32, 0.0, Bd.KERNEL_TMA)
        torch.cuda.synchronize()
        barrier(world)
        stage = [torch.empty(5, dtype=torch.float64).pin_memory() for _ in range(2)]
        t0 = time.perf_counter()
        g2 = Bd.Grid(p, *(h.numpy() for h in host), stream=stream.cuda_stream)
        # every step's totals are read back; step n+1 is launched before the
        # host waits for the totals of step n, so the GPU does not idle
        prev = None
        bad = 0
        for k in range(args.steps):
            g2.step(1)
            cur = (g2.totals_async(stage[k & 1]), k & 1)
            if prev is not None:
                g2.totals_wait(prev[0])
                bad += int(stage[prev[1]][4].item() != 0.0)
            prev = cur
        g2.totals_wait(prev[0])
        bad += int(stage[prev[1]][4].item() != 0.0)
        g2.macro([o.numpy() for o in outs])
        el = time.perf_counter() - t0
        assert bad == 0
        barrier(world)
        el = allmax(el, world)
        g2.close()
        h2d = 4 * 8 * cells
        d2h = 4 * 8 * cells + 32 * args.steps
        line["e2e"] = {"value": whole_job_rate(cells, args.steps, el * 1e3, world), "unit": "cell-updates/s",
                       "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                       "what": "mrt_create from pinned host rho,u,v,T; per step mrt_step(1) + "
                               "mrt_conserved_totals_async into pinned host memory, waited for one step later "
                               "(mrt_totals_wait); final mrt_get_macro to pinned host"}

    if rank == 0 and world == 1 and not args.no_cpu:
        rate, cores, sample = cpu_oracle_rate(w)
        import oracle
        oracle.set_threads(1)
        rate1, _, sample1 = cpu_oracle_rate(w, budget_s=4.0, rows=64)
        oracle.set_threads(cores)
        line["cpu_baseline"] = {"value": rate, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
                                "sample": sample, "one_core": {"value": rate1, "sample": sample1}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def adjoint_costs(Bd, W, torch, stream, advection=0, cases=None):
    """Forward vs recorded-forward vs reverse-sweep time per step."""
    out = {}
    if cases is None:
        cases = [("smooth_vortex_512x512_fp32", W.smooth_vortex(n=512, nsteps=500), 500, 50),
                 ("kelvin_helmholtz_4096x4096_fp32", W.kelvin_helmholtz(n=4096, nsteps=40), 40, 10)]
    for name, w, nsteps, ck in cases:
        with torch.cuda.stream(stream):
            fields = [torch.tensor(np.ascontiguousarray(a), device="cuda") for a in (w.rho, w.ux, w.uy, w.T)]
            dL = torch.full((w.ny, w.nx), w.dx * w.dx, dtype=torch.float64, device="cuda")
            outs = [torch.empty_like(dL) for _ in range(4)]
        g = Bd.Grid.from_workload(w, precision=Bd.FP32, stream=stream.cuda_stream, advection=advection)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        g.step(5)
        torch.cuda.synchronize()
        e[0].record(stream)
        g.step(nsteps)
        e[1].record(stream)
        torch.cuda.synchronize()
        e[2].record(stream)
        g.adjoint_record(*fields, nsteps, ck)
        e[3].record(stream)
        torch.cuda.synchronize()
        e[4].record(stream)
        g.adjoint_backward(dL, outs)
        e[5].record(stream)
        torch.cuda.synchronize()
        g.close()
        fwd = e[0].elapsed_time(e[1]) / nsteps
        rec = e[2].elapsed_time(e[3]) / nsteps
        bwd = e[4].elapsed_time(e[5]) / nsteps
        out[name] = {"steps": nsteps, "ckpt_every": ck, "forward_ms_per_step": fwd,
                     "record_ms_per_step": rec, "backward_ms_per_step": bwd,
                     "backward_over_forward": bwd / fwd,
                     "note": "device-resident fields and gradients; backward = segment recompute + "
                             "reverse step + ghost/init adjoints + rate sums"}
    return out


def _shock_x(rho, dx, behind, ahead):
    """Position of a right-moving shock: the last cell centre (from the
    right) where rho exceeds the mean of the two states, interpolated."""
    mid = 0.5 * (behind + ahead)
    i = int(np.nonzero(rho > mid)[0][-1])
    x = (i + 0.5) * dx
    if i + 1 < len(rho):
        x += dx * (rho[i] - mid) / (rho[i] - rho[i + 1])
    return x


def paper_problems(Bd, W, torch, stream, peak, cap=0):
    """Sod (400 x 4, FP64), strong shock (2048 x 8, FP32 and FP64), colliding
    shocks (1300 x 4, gamma 7/5, MRT and SRT rates, FP64, t = 0.13), the
    Richtmyer-Meshkov run (360 x 100, reflecting wall, t = 0.104) and the
    four-quadrant 2-D Riemann problem (500^2): cell-updates/s with the error
    against the stored exact solutions where one exists.  cap > 0: at most
    cap steps per problem, timings only."""
    with open(EXACT_PROFILES) as fh:
        exact = json.load(fh)
    out = {}
    if cap > 0:
        cases = [("sod_400x4", W.sod_tube(), (Bd.FP64,)), ("strong_shock_2048x8", W.strong_shock(), (Bd.FP32, Bd.FP64)),
                 ("colliding_shocks_gamma1.4", W.colliding_shocks(gamma=1.4), (Bd.FP64,)),
                 ("richtmyer_meshkov_360x100", W.richtmyer_meshkov(), (Bd.FP32, Bd.FP64)),
                 ("four_quadrant_500x500", W.four_quadrant_riemann(n=500), (Bd.FP32,))]
        for name, w, precs in cases:
            n = min(cap, w.nsteps)
            for prec in precs:
                g = Bd.Grid.from_workload(w, precision=prec, stream=stream.cuda_stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                e0.record(stream)
                g.step(n)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                out[f"{name}_{'fp64' if prec == Bd.FP64 else 'fp32'}"] = {
                    "steps": n, "ms": ms, "us_per_step": 1e3 * ms / n, "kernel": g.info()["kernel"],
                    "healthy": g.health() == Bd.MRT_OK}
                g.close()
        return out

    def timed(w, prec, nsteps):
        g = Bd.Grid.from_workload(w, precision=prec, stream=stream.cuda_stream)
        t0 = g.totals()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        return g, ms, t0

    cases = [("sod_400x4", W.sod_tube(), (Bd.FP64,)), ("strong_shock_2048x8", W.strong_shock(), (Bd.FP32, Bd.FP64)),
             ("colliding_shocks_gamma1.4", W.colliding_shocks(gamma=1.4), (Bd.FP64,)),
             ("colliding_shocks_gamma1.4_srt", W.colliding_shocks(gamma=1.4, mrt=False), (Bd.FP64,))]
    def hbm(prec, rate):
        # algorithmic bytes (16 reads + 16 writes per cell-update) per second
        # over the measured copy peak
        return (BYTES_PER_CELL_F64 if prec == Bd.FP64 else BYTES_PER_CELL_F32) * rate / 1e9 / peak

    for name, w, precs in cases:
        ex = exact[name.replace("_srt", "")]
        rho_ex = np.asarray(ex["rho"])
        for prec in precs:
            g, ms, t0 = timed(w, prec, w.nsteps)
            ok = g.health() == Bd.MRT_OK
            r = g.macro()[0][0]
            t1 = g.totals()
            g.close()
            rate = w.cells * w.nsteps / (ms * 1e-3)
            d = {"steps": w.nsteps, "ms": ms, "cell_updates_per_s": rate, "hbm_frac": hbm(prec, rate),
                 "healthy": ok, "l1_rho_vs_exact": float(np.mean(np.abs(r - rho_ex))),
                 "tv_excess": float(np.sum(np.abs(np.diff(r))) - np.sum(np.abs(np.diff(rho_ex))))}
            if not name.startswith("colliding"):
                # u = 0 at both fixed ends: the total mass is conserved
                d["mass_drift_rel"] = float(abs(t1[0] - t0[0]) / abs(t0[0]))
                d["shock_x_error_dx"] = (_shock_x(r, w.dx, ex["star"]["rho_r"], ex["right"][0])
                                         - ex["shock_x"]["right"]) / w.dx
            out[f"{name}_{'fp64' if prec == Bd.FP64 else 'fp32'}"] = d
    w = W.four_quadrant_riemann(n=500, nsteps=1000)
    g, ms, _ = timed(w, Bd.FP32, 1000)
    flagged = None
    for k in range(1000, 12000, 100):
        if g.health() != Bd.MRT_OK:
            flagged = k
            break
        g.step(100)
    g.close()
    wr = W.richtmyer_meshkov()
    for prec in (Bd.FP32, Bd.FP64):
        g, ms_rm, _ = timed(wr, prec, wr.nsteps)
        ok = g.health() == Bd.MRT_OK
        r = g.macro()[0]
        g.close()
        rate = wr.cells * wr.nsteps / (ms_rm * 1e-3)
        out[f"richtmyer_meshkov_360x100_{'fp64' if prec == Bd.FP64 else 'fp32'}"] = {
            "steps": wr.nsteps, "ms": ms_rm, "cell_updates_per_s": rate, "hbm_frac": hbm(prec, rate),
            "healthy": ok, "y_symmetry_max_rel": float(np.max(np.abs(r - r[::-1])) / np.max(r)),
            "rho_range": [float(r.min()), float(r.max())]}
    out["four_quadrant_500x500_fp32"] = {"steps": 1000, "ms": ms,
                                         "cell_updates_per_s": w.cells * 1000 / (ms * 1e-3),
                                         "hbm_frac": hbm(Bd.FP32, w.cells * 1000 / (ms * 1e-3)),
                                         "health_flag_by_step": flagged,
                                         "note": "positivity of P is lost near step 1400 under forward Euler"}
    return out


def batch_sweep(Bd, W, torch, args, peak):
    """The 256-instance sweep (oracle-screened draws, FP32): autotuned kernel
    variant and work-item height, then K timed steps of every instance
    (graph replays on the batch's stream, CUDA events on that stream)."""
    from paper_1004_5442_gb300 import autotune as AT
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "tests", "golden", "riemann_instances_screened.json")) as fh:
        screened = json.load(fh)
    ws = W.riemann_instances(count=args.batch_count, accepted=screened["accepted"])
    cells = sum(w.nx * w.ny for w in ws)
    t0 = time.perf_counter()
    tuned = AT.tune_workloads(ws, use_cache=False)
    tune_s = time.perf_counter() - t0
    with Bd.Batch(ws) as b:
        b.tune(tuned["tile"], tuned["rows_per_item"])
        info = b.info()
        st = torch.cuda.ExternalStream(b.stream)
        b.step(3)
        b.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = args.batch_steps
        e0.record(st)
        b.step(k)
        e1.record(st)
        torch.cuda.synchronize()
        b.sync()
        ms = e0.elapsed_time(e1)
        healthy = sum(b.grid(i).health() == Bd.MRT_OK for i in range(len(ws)))
    per_s = ms * 1e-3 / k
    gbs = BYTES_PER_CELL_F32 * cells / per_s / 1e9
    return {"workload": f"riemann_ripple_sweep_{len(ws)}_fp32", "instances": len(ws), "cells": cells,
            "value": cells / per_s, "unit": "cell-updates/s", "steps": k, "ms_per_step": ms / k,
            "hbm_achieved_gbs": gbs, "hbm_frac": gbs / peak, "launches_per_step": 1,
            "tile": info["tile"], "rows_per_item": info["rows_per_item"], "ctas": info["ctas"],
            "work_items": info["items"], "autotune_s": tune_s,
            "autotune": [(d["tile"], d["rows_per_item"], round(d["ms_per_step"], 4)) for d in tuned["timings"]],
            "healthy_after": {"steps": k + 3, "instances_ok": healthy},
            "screening": {"acceptance_rate": screened["acceptance_rate"],
                          "rule": "FP64 oracle on the full instance: rho and T finite and positive after each of "
                                  "1000 steps"}}


def sweep_tiles(args):
    """Time every compiled TMA variant on the workload (tuning aid)."""
    import torch
    from paper_1004_5442_gb300 import build as B
    B.build()
    from paper_1004_5442_gb300 import binding as Bd
    from paper_1004_5442_gb300 import workloads as W
    w = W.kelvin_helmholtz(n=args.n, nsteps=0)
    for prec in (Bd.FP32, Bd.FP64):
        for tile in (1, 2, 3, 4, 5, 6, 7):
            g = Bd.Grid.from_workload(w, precision=prec, kernel=Bd.KERNEL_TMA, tile=tile)
            g.step(max(args.warmup, 3))
            k = args.steps if prec == Bd.FP32 else max(5, args.steps // 10)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.step(k)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            bpc = 128 if prec == Bd.FP32 else 256
            print(json.dumps({"tile": tile, "precision": "fp32" if prec == Bd.FP32 else "fp64",
                              "ms_per_step": ms, "cell_updates_per_s": w.cells / (ms * 1e-3),
                              "hbm_gbs": bpc * w.cells / (ms * 1e-3) / 1e9}), flush=True)
            g.close()


def fma_only(args):
    """The device's multiply-add throughput, FP64 and FP32, at 2, 4 and 8
    blocks of 256 threads per SM, three launches each (CUDA events inside
    mrt_debug_fma_rate)."""
    import torch
    from paper_1004_5442_gb300 import build as B
    B.build()
    from paper_1004_5442_gb300 import binding as Bd
    out = {}
    for name, prec in (("fp64", Bd.FP64), ("fp32", Bd.FP32)):
        for bps in (2, 4, 8):
            runs = [Bd.fma_rate(prec, blocks_per_sm=bps) for _ in range(3)]
            out[f"{name}_blocks_per_sm_{bps}"] = {"tflops": [r / 1e12 for r, _ in runs], "ms": [m for _, m in runs]}
    # FP64 with few warps: one block per SM of 1 or 4 warps, 32 down to 1
    # active lanes; clocks per warp multiply-add per SM at the observed rate
    clk = 2.07e9
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for warps in (1, 4):
        for lanes in (32, 8, 1):
            r, ms = Bd.fma_rate(Bd.FP64, iters=1250, blocks_per_sm=1, threads_per_block=32 * warps, active_lanes=lanes)
            warp_fma = r / 2 / lanes                     # warp multiply-adds per second
            out[f"fp64_warps_per_sm_{warps}_lanes_{lanes}"] = {"tflops": r / 1e12, "ms": ms,
                                                               "clocks_per_warp_fma_per_sm": clk * sms / warp_fma}
    for blocks in (1, 152, 608):
        a, b = Bd.launch_period(2000, blocks, 128)
        out[f"launch_period_{blocks}_blocks_of_128"] = {"us_stream": a, "us_graph_of_two": b}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.sweep_tiles:
        sweep_tiles(args)
        return
    if args.fma_only:
        fma_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
