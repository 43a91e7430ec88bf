"""mrt_conserved_totals_static: conserved totals of a caller-held device
state with the scratch in a fixed array of the library instead of memory
the library allocates.  It serves callers that cannot allocate device memory
when they need the totals: a framework that owns the device-memory budget
through its own pool, or a monitoring loop that must not stall on the
allocator (cudaMalloc and cudaFree can synchronise the device).  Its result is
checked against the grid entry point mrt_conserved_totals on the same state,
on two calls in a row, with the tolerances of the other totals tests.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import build as B
from paper_1004_5442_gb300 import workloads as W


def _abs_scale(f, dx):
    """sum over cells of |moment k| * dx^2 for k = 1..4 (the scale of each
    total), from a device state, a few rows at a time."""
    import torch
    import oracle
    _, _, _, M, _ = oracle.model()
    Mt = torch.tensor(M[:4], dtype=torch.float64, device=f.device)
    out = torch.zeros(4, dtype=torch.float64, device=f.device)
    for y0 in range(0, f.shape[1], 512):
        chunk = f[:, y0:y0 + 512, :].double()
        out += torch.einsum("ki,iyx->kyx", Mt, chunk).abs().sum(dim=(1, 2))
    return out.cpu().numpy() * dx * dx


# 300 x 37: one partial block; 1000 x 300: 19 blocks with a ragged last one;
# 8192 x 8192: the largest grid the fixed scratch takes (4096 blocks)
CASES = [(300, 37, Bd.FP64, 1e-13), (300, 37, Bd.FP32, 1e-5), (1000, 300, Bd.FP64, 1e-13),
         (1000, 300, Bd.FP32, 1e-5), (8192, 8192, Bd.FP32, 1e-5)]


@pytest.mark.gpu
@pytest.mark.parametrize("nx,ny,prec,tol", CASES)
def test_static_totals_match_grid_totals(nx, ny, prec, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    dtype = torch.float64 if prec == Bd.FP64 else torch.float32
    w = W.random_smooth(nx, ny, seed=12, amp=0.1)
    with Bd.Grid.from_workload(w, precision=prec) as g:
        for call in range(2):                     # two calls in a row, different states
            g.step(3 + 2 * call)
            want = g.totals()                     # existing entry point
            f = torch.empty((16, w.ny, w.nx), dtype=dtype, device="cuda")
            g.get_f(out=f)
            torch.cuda.synchronize()
            out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            Bd.conserved_totals_static(f, prec, w.nx, w.ny, w.dx, out,
                                       stream=torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            scale = _abs_scale(f, w.dx)
            del f
            assert np.all(np.isfinite(got))
            assert np.all(np.abs(got - want) <= tol * scale), (call, got, want)


def test_static_totals_rejects_oversized_grid():
    B.build()
    L = Bd.load()
    import ctypes
    rc = L.mrt_conserved_totals_static(ctypes.c_void_p(16), Bd.FP32, 8193, 8192, 1.0,
                                       ctypes.c_void_p(16), None)
    assert rc == Bd.MRT_EINVAL
    assert "exceeds the fixed scratch capacity" in L.mrt_last_error().decode()
