"""ctypes binding of the C ABI in include/mrtfdlb.h (argument marshalling only).

Every step of the method runs in the CUDA library; this module converts
numpy arrays / torch tensors to pointers, passes torch's current CUDA stream,
and turns error codes into exceptions.  If the compiled library is missing
the import fails loudly: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmrtfdlb.so")

MRT_OK, MRT_EINVAL, MRT_ENOMEM, MRT_ECUDA, MRT_EUNSTABLE, MRT_ETIMEOUT = range(6)
FP32, FP64 = 0, 1
BC_PERIODIC, BC_FIXED_EQ, BC_REFLECT_FIXED = 0, 1, 2
KERNEL_AUTO, KERNEL_TMA, KERNEL_DIRECT, KERNEL_SPLIT = 0, 1, 2, 3
ADV_LW, ADV_LW2D = 0, 1

# every symbol include/mrtfdlb.h declares
EXPORTED = ["mrt_create", "mrt_step", "mrt_get_macro", "mrt_conserved_totals", "mrt_get_f",
            "mrt_set_f", "mrt_health", "mrt_info", "mrt_destroy", "mrt_status_str",
            "mrt_last_error", "mrt_conserved_totals_static", "mrt_adjoint_record",
            "mrt_adjoint_backward", "mrt_adjoint_step", "mrt_batch_create", "mrt_batch_step",
            "mrt_batch_tune", "mrt_batch_grid", "mrt_batch_info", "mrt_batch_sync", "mrt_batch_stream",
            "mrt_batch_destroy", "mrt_debug_padding", "mrt_debug_wait_timeout", "mrt_conserved_totals_async",
            "mrt_totals_wait", "mrt_save", "mrt_load", "mrt_debug_fma_rate", "mrt_debug_launch_period"]


class MrtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


_STATUS = {MRT_OK: "MRT_OK", MRT_EINVAL: "MRT_EINVAL", MRT_ENOMEM: "MRT_ENOMEM",
           MRT_ECUDA: "MRT_ECUDA", MRT_EUNSTABLE: "MRT_EUNSTABLE", MRT_ETIMEOUT: "MRT_ETIMEOUT"}


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double),
                ("dt", ctypes.c_double), ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
                ("s", ctypes.c_double * 16), ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
                ("precision", ctypes.c_int), ("kernel", ctypes.c_int), ("tile", ctypes.c_int),
                ("advection", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libmrtfdlb.so (built by paper_1004_5442_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run paper_1004_5442_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.mrt_create.argtypes = [ctypes.POINTER(Params), vp, vp, vp, vp, ip, vp, ctypes.POINTER(vp)]
    L.mrt_step.argtypes = [vp, ctypes.c_long]
    L.mrt_get_macro.argtypes = [vp, vp, vp, vp, vp, ip]
    L.mrt_conserved_totals.argtypes = [vp, dp]
    L.mrt_get_f.argtypes = [vp, vp, ip]
    L.mrt_set_f.argtypes = [vp, vp, ip]
    L.mrt_health.argtypes = [vp]
    L.mrt_info.argtypes = [vp, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long),
                           ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)]
    L.mrt_destroy.argtypes = [vp]
    L.mrt_destroy.restype = None
    L.mrt_status_str.restype = ctypes.c_char_p
    L.mrt_status_str.argtypes = [ip]
    L.mrt_last_error.restype = ctypes.c_char_p
    L.mrt_conserved_totals_static.argtypes = [vp, ip, ip, ip, ctypes.c_double, vp, vp]
    L.mrt_adjoint_record.argtypes = [vp, vp, vp, vp, vp, ip, ctypes.c_long, ip]
    L.mrt_adjoint_backward.argtypes = [vp, vp, ip, vp, vp, vp, vp, dp]
    L.mrt_adjoint_step.argtypes = [vp, vp, vp, vp, ip, dp]
    vpp = ctypes.POINTER(ctypes.c_void_p)
    L.mrt_batch_create.argtypes = [ip, ctypes.POINTER(Params), vpp, vpp, vpp, vpp, ip, ctypes.POINTER(vp)]
    L.mrt_batch_step.argtypes = [vp, ctypes.c_long]
    L.mrt_batch_tune.argtypes = [vp, ip, ip]
    L.mrt_batch_grid.argtypes = [vp, ip, ctypes.POINTER(vp)]
    ipp = ctypes.POINTER(ctypes.c_int)
    L.mrt_batch_info.argtypes = [vp, ipp, ipp, ipp, ipp, ipp]
    L.mrt_batch_sync.argtypes = [vp]
    L.mrt_batch_stream.argtypes = [vp, ctypes.POINTER(vp)]
    L.mrt_debug_padding.argtypes = [vp, ctypes.POINTER(ctypes.c_long)]
    L.mrt_debug_wait_timeout.argtypes = [vp]
    L.mrt_conserved_totals_async.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_long)]
    L.mrt_totals_wait.argtypes = [vp, ctypes.c_long]
    L.mrt_save.argtypes = [vp, ctypes.c_char_p]
    L.mrt_load.argtypes = [vp, ctypes.c_char_p]
    L.mrt_debug_fma_rate.argtypes = [ip, ctypes.c_long, ip, ip, ip, dp, dp]
    L.mrt_debug_launch_period.argtypes = [ip, ip, ip, dp, dp]
    L.mrt_batch_destroy.argtypes = [vp]
    L.mrt_batch_destroy.restype = None
    for name in ("mrt_create", "mrt_step", "mrt_get_macro", "mrt_conserved_totals", "mrt_get_f",
                 "mrt_set_f", "mrt_health", "mrt_info", "mrt_conserved_totals_static",
                 "mrt_adjoint_record", "mrt_adjoint_backward", "mrt_adjoint_step", "mrt_batch_create",
                 "mrt_batch_step", "mrt_batch_tune", "mrt_batch_grid", "mrt_batch_info", "mrt_batch_sync",
                 "mrt_batch_stream", "mrt_debug_padding", "mrt_debug_wait_timeout", "mrt_conserved_totals_async",
                 "mrt_totals_wait", "mrt_save", "mrt_load", "mrt_debug_fma_rate", "mrt_debug_launch_period"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(code: int) -> None:
    if code != MRT_OK:
        raise MrtError(code, load().mrt_last_error().decode())


def _ptr(a) -> int:
    """Address of a C-contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return a.ctypes.data
    assert a.is_contiguous(), "tensor must be contiguous"
    return a.data_ptr()


def _on_device(a) -> int:
    return int(not isinstance(a, np.ndarray) and a.is_cuda)


def _torch_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def make_params(nx, ny, dx, dt, gamma, s, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC, precision=FP32,
                Pr=0.0, kernel=KERNEL_AUTO, tile=0, advection=0) -> Params:
    p = Params()
    p.nx, p.ny, p.dx, p.dt, p.gamma, p.Pr = int(nx), int(ny), float(dx), float(dt), float(gamma), float(Pr)
    for k in range(16):
        p.s[k] = float(s[k])
    p.bc_x, p.bc_y, p.precision, p.kernel = int(bc_x), int(bc_y), int(precision), int(kernel)
    p.tile = int(tile)
    p.advection = int(advection)
    return p


def conserved_totals_static(f, precision: int, nx: int, ny: int, dx: float, out, stream=None) -> None:
    """Totals of a dense [16][ny][nx] device state into out (4 doubles on the
    device) without any allocation by the library (mrt_conserved_totals_static)."""
    if stream is None:
        stream = _torch_stream()
    check(load().mrt_conserved_totals_static(ctypes.c_void_p(_ptr(f)), int(precision), int(nx), int(ny),
                                             float(dx), ctypes.c_void_p(_ptr(out)), ctypes.c_void_p(stream)))


def fma_rate(precision: int, iters: int | None = None, blocks_per_sm: int = 4, threads_per_block: int = 256,
             active_lanes: int = 32):
    """(flop/s, ms) of the device's fused multiply-add throughput in FP32 or
    FP64 (mrt_debug_fma_rate); iters defaults to about 0.1 s of work at
    full occupancy."""
    if iters is None:
        iters = 3000 if precision == FP64 else 200000
    rate, ms = ctypes.c_double(), ctypes.c_double()
    check(load().mrt_debug_fma_rate(int(precision), int(iters), int(blocks_per_sm), int(threads_per_block),
                                    int(active_lanes), ctypes.byref(rate), ctypes.byref(ms)))
    return rate.value, ms.value


def launch_period(nlaunches: int = 2000, blocks: int = 1, threads: int = 128):
    """(us per launch on a stream, us per launch in two-launch CUDA graphs)
    of a kernel that does nothing (mrt_debug_launch_period)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    check(load().mrt_debug_launch_period(int(nlaunches), int(blocks), int(threads), ctypes.byref(a),
                                         ctypes.byref(b)))
    return a.value, b.value


class Grid:
    """A grid owned by the CUDA library (handle wrapper)."""

    def __init__(self, params: Params, rho, ux, uy, T, stream=None):
        L = load()
        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.fp64 = params.precision == FP64
        arrs = [rho, ux, uy, T]
        dev = {_on_device(a) for a in arrs}
        if len(dev) != 1:
            raise ValueError("fields must all be on the host or all on the device")
        on_dev = dev.pop()
        if not on_dev:
            arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64),
                                                         (self.ny, self.nx))) for a in arrs]
        if stream is None:
            stream = _torch_stream() if on_dev else 0
        self.stream = stream
        h = ctypes.c_void_p()
        check(L.mrt_create(ctypes.byref(params), *(ctypes.c_void_p(_ptr(a)) for a in arrs),
                           on_dev, ctypes.c_void_p(stream), ctypes.byref(h)))
        self._h = h

    @classmethod
    def view(cls, handle, nx, ny, fp64=False):
        """A non-owning wrapper of a grid handle (e.g. a batch instance)."""
        g = cls.__new__(cls)
        g._h = ctypes.c_void_p(handle)
        g.nx, g.ny, g.fp64 = nx, ny, fp64
        g._owned = False
        return g

    @classmethod
    def from_workload(cls, w, precision=FP32, kernel=KERNEL_AUTO, stream=None, tile=0, advection=0):
        p = make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, w.s, w.bc_x, w.bc_y, precision, 0.0, kernel, tile,
                        advection)
        return cls(p, w.rho, w.ux, w.uy, w.T, stream=stream)

    @property
    def handle(self):
        return self._h

    def step(self, n: int = 1) -> None:
        check(load().mrt_step(self._h, int(n)))

    def macro(self, out=None):
        """(rho, ux, uy, T) as float64 numpy arrays (or into given device tensors)."""
        if out is None:
            out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        check(load().mrt_get_macro(self._h, *(ctypes.c_void_p(_ptr(o)) for o in out),
                                   _on_device(out[0])))
        return tuple(out)

    def totals(self) -> np.ndarray:
        out = np.zeros(4)
        check(load().mrt_conserved_totals(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def totals_async(self, dst) -> int:
        """Enqueue the totals and flag word into dst (5 doubles of page-locked
        host memory: a pinned torch tensor or a numpy view of one); returns the
        ticket to pass to totals_wait (mrt_conserved_totals_async)."""
        t = ctypes.c_long()
        check(load().mrt_conserved_totals_async(self._h, ctypes.c_void_p(_ptr(dst)), ctypes.byref(t)))
        return t.value

    def totals_wait(self, ticket: int) -> None:
        check(load().mrt_totals_wait(self._h, int(ticket)))

    def save(self, path) -> None:
        """Write the state, fixed ghosts and step count to a file (mrt_save)."""
        check(load().mrt_save(self._h, os.fsencode(path)))

    def load(self, path) -> None:
        """Restore a state written by save into this matching grid (mrt_load)."""
        check(load().mrt_load(self._h, os.fsencode(path)))

    def get_f(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((16, self.ny, self.nx), dtype=np.float64 if self.fp64 else np.float32)
        check(load().mrt_get_f(self._h, ctypes.c_void_p(_ptr(out)), _on_device(out)))
        return out

    def set_f(self, f) -> None:
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64 if self.fp64 else np.float32)
        check(load().mrt_set_f(self._h, ctypes.c_void_p(_ptr(f)), _on_device(f)))

    def adjoint_record(self, rho0, ux0, uy0, T0, nsteps: int, ckpt_every: int) -> None:
        """Set f = f^eq(fields), run nsteps keeping checkpoints (mrt_adjoint_record)."""
        arrs = [rho0, ux0, uy0, T0]
        on_dev = _on_device(arrs[0])
        if not on_dev:
            arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (self.ny, self.nx)))
                    for a in arrs]
        check(load().mrt_adjoint_record(self._h, *(ctypes.c_void_p(_ptr(a)) for a in arrs), on_dev,
                                        int(nsteps), int(ckpt_every)))

    def adjoint_backward(self, dL_drhoN, outs=None):
        """(g_rho0, g_ux0, g_uy0, g_T0, g_s[16]) from dL/drho_N (mrt_adjoint_backward)."""
        on_dev = _on_device(dL_drhoN)
        if not on_dev:
            dL_drhoN = np.ascontiguousarray(dL_drhoN, dtype=np.float64)
        if outs is None:
            outs = [np.empty((self.ny, self.nx)) for _ in range(4)]
        gs = np.zeros(16)
        check(load().mrt_adjoint_backward(self._h, ctypes.c_void_p(_ptr(dL_drhoN)), on_dev,
                                          *(ctypes.c_void_p(_ptr(o)) for o in outs),
                                          gs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return (*outs, gs)

    def adjoint_step(self, f, lam_next):
        """One reverse step on host states: returns (dL/df^n, dL/ds of this step)."""
        dt = np.float64 if self.fp64 else np.float32
        f = np.ascontiguousarray(f, dtype=dt)
        lam_next = np.ascontiguousarray(lam_next, dtype=dt)
        lam = np.empty_like(f)
        gs = np.zeros(16)
        check(load().mrt_adjoint_step(self._h, ctypes.c_void_p(_ptr(f)), ctypes.c_void_p(_ptr(lam_next)),
                                      ctypes.c_void_p(_ptr(lam)), 0,
                                      gs.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return lam, gs

    def health(self) -> int:
        return int(load().mrt_health(self._h))

    def debug_padding(self) -> int:
        """Nonzero words in the never-written padding columns (0 = no stray writes)."""
        n = ctypes.c_long()
        check(load().mrt_debug_padding(self._h, ctypes.byref(n)))
        return n.value

    def debug_wait_timeout(self) -> None:
        """Let a bounded device wait run out; mrt_health then reports MRT_ETIMEOUT."""
        check(load().mrt_debug_wait_timeout(self._h))

    def info(self) -> dict:
        steps, pitch, plane = ctypes.c_long(), ctypes.c_long(), ctypes.c_long()
        kern, tile = ctypes.c_int(), ctypes.c_int()
        check(load().mrt_info(self._h, ctypes.byref(steps), ctypes.byref(pitch), ctypes.byref(plane),
                              ctypes.byref(kern), ctypes.byref(tile)))
        return {"steps": steps.value, "pitch": pitch.value, "plane": plane.value,
                "kernel": kern.value, "tile": tile.value}

    def close(self) -> None:
        if not getattr(self, "_owned", True):
            return
        if getattr(self, "_h", None) is not None and self._h.value:
            load().mrt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Independent FP32 grids advanced together (mrt_batch_*)."""

    def __init__(self, workloads, fields_on_device=False):
        L = load()
        n = len(workloads)
        params = (Params * n)()
        self.shapes = []
        keep = []
        ptrs = [(ctypes.c_void_p * n)() for _ in range(4)]
        for i, w in enumerate(workloads):
            params[i] = make_params(w.nx, w.ny, w.dx, w.dt, w.gamma, w.s, w.bc_x, w.bc_y, FP32)
            arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (w.ny, w.nx)))
                    for a in (w.rho, w.ux, w.uy, w.T)]
            keep.append(arrs)
            for q in range(4):
                ptrs[q][i] = arrs[q].ctypes.data
            self.shapes.append((w.nx, w.ny))
        h = ctypes.c_void_p()
        check(L.mrt_batch_create(n, params, *(ctypes.cast(p, ctypes.POINTER(ctypes.c_void_p)) for p in ptrs),
                                 0, ctypes.byref(h)))
        self._h = h
        self.n = n

    def step(self, n: int = 1) -> None:
        check(load().mrt_batch_step(self._h, int(n)))

    def tune(self, tile: int, rows_per_item: int) -> None:
        check(load().mrt_batch_tune(self._h, int(tile), int(rows_per_item)))

    def sync(self) -> None:
        check(load().mrt_batch_sync(self._h))

    @property
    def stream(self) -> int:
        """Raw cudaStream_t the batch launches on (for events)."""
        h = ctypes.c_void_p()
        check(load().mrt_batch_stream(self._h, ctypes.byref(h)))
        return h.value or 0

    def info(self) -> dict:
        v = [ctypes.c_int() for _ in range(5)]
        check(load().mrt_batch_info(self._h, *(ctypes.byref(x) for x in v)))
        return dict(zip(("n", "tile", "rows_per_item", "ctas", "items"), (x.value for x in v)))

    def grid(self, i: int) -> Grid:
        h = ctypes.c_void_p()
        check(load().mrt_batch_grid(self._h, int(i), ctypes.byref(h)))
        nx, ny = self.shapes[i]
        return Grid.view(h.value, nx, ny, False)

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            load().mrt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
