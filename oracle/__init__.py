"""FP64 CPU oracle for the D2V16 thermal MRT finite-difference LB step.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package; the GPU library never does.  The arithmetic lives in
``mrt_oracle.c`` (plain C, FP64, dense 16x16 loops) and in ``riemann.py``
(exact Riemann solution used as a pin); this module only compiles the C file
with gcc and marshals numpy arrays through ctypes.

Layout of every distribution array: ``f[i, y, x]`` (16, ny, nx), float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

BC_PERIODIC = 0
BC_FIXED_EQ = 1
BC_REFLECT_FIXED = 2   # reflecting wall at the low end, fixed-equilibrium inflow at the high end
# space discretisation: the paper's Lax-Wendroff operator axis by axis (ADV_LW),
# the unsplit 2-D Lax-Wendroff operator with the mixed term (ADV_LW2D), or a
# flux-limited variant (first-order upwind flux plus the Lax-Wendroff
# correction scaled by a limiter; outside the paper)
ADV_LW = 0
ADV_LW2D = 1
ADV_MINMOD = 2
ADV_VANLEER = 3
# another reading of the time scheme: the Lax-Wendroff (second-order Taylor)
# step of the whole kinetic equation, collision term included (forward only)
ADV_LWFULL = 4
NV = 16


def build(force: bool = False) -> str:
    """Compile ``mrt_oracle.c`` into ``oracle/_build/liboracle.so`` with gcc.

    IEEE semantics are kept: no fast-math and no FMA contraction, so the
    oracle gives the same bits on x86-64 and aarch64 hosts.
    """
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double),
                ("b", ctypes.c_double), ("s", ctypes.c_double * NV),
                ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int), ("advection", ctypes.c_int)]


_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_model.argtypes = [dp, dp, dp, dp, dp]
        L.orc_invert.argtypes = [dp, dp, ctypes.c_int]
        L.orc_invert.restype = ctypes.c_int
        L.orc_feq_moments.argtypes = [ctypes.c_double] * 5 + [dp]
        L.orc_feq.argtypes = [ctypes.c_double] * 5 + [dp]
        L.orc_init.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp]
        L.orc_ghosts_from_initial.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_step.argtypes = [ctypes.POINTER(_Cfg), dp, dp, dp, dp]
        L.orc_run.argtypes = [ctypes.POINTER(_Cfg), dp, dp, dp, ctypes.c_long, dp]
        L.orc_macro.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, dp]
        L.orc_totals.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
        L.orc_feq_jacobian.argtypes = [ctypes.c_double] * 5 + [dp]
        L.orc_feq_moments_via_cplx.argtypes = [ctypes.c_double] * 5 + [dp]
        L.orc_step_adjoint.argtypes = [ctypes.POINTER(_Cfg), dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_init_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double] + [dp] * 9
        L.orc_ghosts_adjoint.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def model():
    """Return (vx, vy, eta2, M, Minv) as built by the oracle (float64)."""
    vx, vy, e2 = (np.zeros(NV) for _ in range(3))
    M = np.zeros((NV, NV))
    Mi = np.zeros((NV, NV))
    lib().orc_model(_p(vx), _p(vy), _p(e2), _p(M), _p(Mi))
    return vx, vy, e2, M, Mi


def invert(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.zeros_like(A)
    if lib().orc_invert(_p(A), _p(out), A.shape[0]) != 0:
        raise np.linalg.LinAlgError("singular")
    return out


def feq_moments(rho, jx, jy, e, b) -> np.ndarray:
    out = np.zeros(NV)
    lib().orc_feq_moments(float(rho), float(jx), float(jy), float(e), float(b), _p(out))
    return out


def feq(rho, ux, uy, T, b) -> np.ndarray:
    out = np.zeros(NV)
    lib().orc_feq(float(rho), float(ux), float(uy), float(T), float(b), _p(out))
    return out


def b_of_gamma(gamma: float) -> float:
    """gamma = (b+2)/b  =>  b = 2/(gamma-1)."""
    return 2.0 / (gamma - 1.0)


@dataclass
class Grid:
    """Oracle state: f (16, ny, nx) plus fixed-equilibrium ghosts."""
    nx: int
    ny: int
    dx: float
    dt: float
    b: float
    s: np.ndarray
    bc_x: int = BC_PERIODIC
    bc_y: int = BC_PERIODIC
    advection: int = ADV_LW
    f: np.ndarray = field(default=None, repr=False)
    gx: np.ndarray = field(default=None, repr=False)
    gy: np.ndarray = field(default=None, repr=False)

    def cfg(self) -> _Cfg:
        c = _Cfg()
        c.nx, c.ny, c.dx, c.dt, c.b = self.nx, self.ny, self.dx, self.dt, self.b
        for k in range(NV):
            c.s[k] = float(self.s[k])
        c.bc_x, c.bc_y = int(self.bc_x), int(self.bc_y)
        c.advection = int(self.advection)
        return c


def create(nx, ny, dx, dt, b, s, rho, ux, uy, T, bc_x=BC_PERIODIC, bc_y=BC_PERIODIC,
           advection=ADV_LW) -> Grid:
    """Initial state f = M^-1 fhat^eq(rho, u, T) and its fixed ghosts."""
    g = Grid(nx, ny, float(dx), float(dt), float(b), np.asarray(s, dtype=np.float64),
             bc_x, bc_y, int(advection))
    arr = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (ny, nx)))
           for a in (rho, ux, uy, T)]
    g.f = np.zeros((NV, ny, nx))
    lib().orc_init(nx, ny, g.b, *(_p(a) for a in arr), _p(g.f))
    g.gx = np.zeros((NV, 2, ny))
    g.gy = np.zeros((NV, 2, nx))
    lib().orc_ghosts_from_initial(nx, ny, _p(g.f), _p(g.gx), _p(g.gy))
    return g


def step(g: Grid, f: np.ndarray | None = None) -> np.ndarray:
    """One step of ``f`` (default g.f); returns the new array (g unchanged)."""
    src = g.f if f is None else np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(src)
    c = g.cfg()
    lib().orc_step(ctypes.byref(c), _p(src), _p(g.gx), _p(g.gy), _p(out))
    return out


def run(g: Grid, nsteps: int) -> Grid:
    """Advance g.f in place by nsteps."""
    work = np.zeros_like(g.f)
    c = g.cfg()
    lib().orc_run(ctypes.byref(c), _p(g.f), _p(g.gx), _p(g.gy), int(nsteps), _p(work))
    return g


def macro(g: Grid, f: np.ndarray | None = None):
    src = g.f if f is None else np.ascontiguousarray(f, dtype=np.float64)
    out = [np.zeros((g.ny, g.nx)) for _ in range(4)]
    lib().orc_macro(g.nx, g.ny, g.b, _p(src), *(_p(o) for o in out))
    return tuple(out)


def totals(g: Grid, f: np.ndarray | None = None) -> np.ndarray:
    src = g.f if f is None else np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_totals(g.nx, g.ny, g.dx, _p(src), _p(out))
    return out


# ---------------------------------------------------------------------------
# Reverse mode
# ---------------------------------------------------------------------------
def feq_jacobian(rho, jx, jy, e, b) -> np.ndarray:
    """d fhat^eq_k / d (rho, jx, jy, e) as a (16, 4) array (complex step)."""
    out = np.zeros(NV * 4)
    lib().orc_feq_jacobian(float(rho), float(jx), float(jy), float(e), float(b), _p(out))
    return out.reshape(NV, 4)


def feq_moments_via_cplx(rho, jx, jy, e, b) -> np.ndarray:
    out = np.zeros(NV)
    lib().orc_feq_moments_via_cplx(float(rho), float(jx), float(jy), float(e), float(b), _p(out))
    return out


def step_adjoint(g: Grid, f: np.ndarray, lam_next: np.ndarray, gxb: np.ndarray, gyb: np.ndarray,
                 gs: np.ndarray) -> np.ndarray:
    """dL/df^n from f^n and dL/df^{n+1}; accumulates ghost and rate adjoints."""
    if g.advection == ADV_LWFULL:
        raise ValueError("ADV_LWFULL has no reverse mode")
    f = np.ascontiguousarray(f, dtype=np.float64)
    lam_next = np.ascontiguousarray(lam_next, dtype=np.float64)
    out = np.zeros_like(f)
    c = g.cfg()
    lib().orc_step_adjoint(ctypes.byref(c), _p(f), _p(g.gx), _p(g.gy), _p(lam_next), _p(out), _p(gxb),
                           _p(gyb), _p(gs))
    return out


def adjoint_run(nx, ny, dx, dt, b, s, rho, ux, uy, T, nsteps, loss_grad, bc_x=BC_PERIODIC,
                bc_y=BC_PERIODIC, ckpt=None, advection=ADV_LW):
    """Gradient of a loss L(rho_N) with respect to the initial fields and the
    16 rates, by reverse mode through nsteps oracle steps.

    loss_grad(rho_N) -> (L, dL/drho_N).  States are kept every `ckpt` steps
    and each segment is recomputed before its reverse sweep.  Returns
    (L, g_rho, g_ux, g_uy, g_T, g_s)."""
    arr = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (ny, nx)))
           for a in (rho, ux, uy, T)]
    g = create(nx, ny, dx, dt, b, s, *arr, bc_x=bc_x, bc_y=bc_y, advection=advection)
    K = nsteps if not ckpt else int(ckpt)
    saved = {}
    f = g.f.copy()
    for n in range(nsteps):
        if n % K == 0:
            saved[n] = f.copy()
        f = step(g, f)
    rhoN = macro(g, f)[0]
    L, dL = loss_grad(rhoN)
    lam = np.ascontiguousarray(np.broadcast_to(np.asarray(dL, dtype=np.float64), (NV, ny, nx)))
    gxb = np.zeros_like(g.gx)
    gyb = np.zeros_like(g.gy)
    gs = np.zeros(NV)
    starts = list(range(0, nsteps, K))
    for s0 in reversed(starts):
        s1 = min(s0 + K, nsteps)
        seg = [saved[s0]]
        for _ in range(s0, s1 - 1):
            seg.append(step(g, seg[-1]))
        for n in reversed(range(s0, s1)):
            lam = step_adjoint(g, seg[n - s0], lam, gxb, gyb, gs)
    lib().orc_ghosts_adjoint(nx, ny, int(bc_x), int(bc_y), _p(gxb), _p(gyb), _p(lam))
    out = [np.zeros((ny, nx)) for _ in range(4)]
    lib().orc_init_adjoint(nx, ny, float(b), *(_p(a) for a in arr), _p(lam), *(_p(o) for o in out))
    return (L, *out, gs)


def forward_loss(nx, ny, dx, dt, b, s, rho, ux, uy, T, nsteps, loss_grad, bc_x=BC_PERIODIC,
                 bc_y=BC_PERIODIC, advection=ADV_LW) -> float:
    """L(rho_N) of a forward oracle run (for finite differences)."""
    g = create(nx, ny, dx, dt, b, s, rho, ux, uy, T, bc_x=bc_x, bc_y=bc_y, advection=advection)
    run(g, nsteps)
    return loss_grad(macro(g)[0])[0]
