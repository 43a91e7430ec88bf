"""torch.autograd.Function over a run of the fused MRT-FDLB step.

``mrt_run(rho0, ux0, uy0, T0, s, params, nsteps, ckpt_every)`` returns the
density after ``nsteps`` steps as a CUDA tensor; its backward runs the CUDA
reverse sweep (mrt_adjoint_backward: checkpointed recomputation + transposed
step) and returns gradients for the four initial fields and the 16 rates.
Only marshalling happens here: every step of the forward and the reverse
sweep runs in the CUDA library.

The recorded run (its checkpoints on the device) belongs to the autograd
graph of the output and is freed with it, so ``backward(retain_graph=True)``
followed by a second backward gives the same gradients again; without
``retain_graph`` a second backward raises PyTorch's usual error.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as Bd


class MRTRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho0, ux0, uy0, T0, s, params, nsteps, ckpt_every):
        p = Bd.make_params(params["nx"], params["ny"], params["dx"], params["dt"], params["gamma"],
                           s.detach().cpu().numpy().astype(np.float64), params.get("bc_x", 0),
                           params.get("bc_y", 0), params.get("precision", Bd.FP32), 0.0,
                           params.get("kernel", Bd.KERNEL_AUTO), params.get("tile", 0),
                           params.get("advection", Bd.ADV_LW))
        fields = [t.detach().to(dtype=torch.float64).contiguous() for t in (rho0, ux0, uy0, T0)]
        grid = Bd.Grid(p, *fields)
        grid.adjoint_record(*fields, nsteps, ckpt_every)
        rhoN = torch.empty_like(fields[0])
        grid.macro([rhoN, torch.empty_like(rhoN), torch.empty_like(rhoN), torch.empty_like(rhoN)])
        ctx.grid = grid
        ctx.save_for_backward(s)
        return rhoN

    @staticmethod
    def backward(ctx, g_rhoN):
        grid = ctx.grid
        (s,) = ctx.saved_tensors
        g = g_rhoN.detach().to(dtype=torch.float64).contiguous()
        outs = [torch.empty_like(g) for _ in range(4)]
        # the reverse sweep runs on the grid's stream: it waits for the work
        # that produced g (and allocated outs) on the caller's stream; the
        # call returns once that stream holds the results
        cur = torch.cuda.current_stream()
        if grid.stream != cur.cuda_stream:
            own = torch.cuda.ExternalStream(grid.stream) if grid.stream else torch.cuda.default_stream()
            own.wait_stream(cur)
        *_, gs = grid.adjoint_backward(g, outs)
        g_s = torch.as_tensor(gs, dtype=s.dtype, device=s.device)
        return outs[0], outs[1], outs[2], outs[3], g_s, None, None, None


def mrt_run(rho0, ux0, uy0, T0, s, params: dict, nsteps: int, ckpt_every: int = 50):
    """rho after nsteps steps from f^eq(rho0, u0, T0), differentiable in all inputs.

    params: nx, ny, dx, dt, gamma, and optionally bc_x, bc_y, precision,
    kernel, tile and advection (Bd.ADV_LW, the method's operator, or
    Bd.ADV_LW2D, the unsplit one)."""
    return MRTRun.apply(rho0, ux0, uy0, T0, s, params, nsteps, ckpt_every)
