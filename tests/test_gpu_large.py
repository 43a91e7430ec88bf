"""A grid far beyond the benchmark size: 16384 x 16384 FP32 (268 M cells,
2 x 17.2 GB of state, the fields built on the device) is stepped by the
automatic kernel choice; after 3 steps, 12 seeded 48^2 windows of step
3 -> 4 (the periodic corners and strip/item seams among them) match one
oracle step on the window, the conserved totals hold and the health flag
stays clear.  Checks that the padded layout, the work-queue item count, the
totals partials and the tensor maps hold up at this size."""
import numpy as np
import pytest

import oracle
from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_16384_squared_fp32_sampled_windows():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    n = 16384
    ref = W.random_smooth(8, 8, seed=1, amp=0.05)       # rates, gamma, CFL convention of the parity cases
    dx = 1.0 / n
    dt = 0.1 * dx / W.V_MAX
    x = (torch.arange(n, device="cuda", dtype=torch.float64) + 0.5) * dx
    X, Y = x[None, :], x[:, None]
    two_pi = 2 * np.pi
    rho = (1 + 0.05 * torch.sin(two_pi * X) * torch.cos(two_pi * 3 * Y)).contiguous()
    ux = (0.1 * torch.cos(two_pi * 2 * Y) + 0 * X).contiguous()
    uy = (0.1 * torch.sin(two_pi * 5 * X) + 0 * Y).contiguous()
    T = (1 + 0.05 * torch.cos(two_pi * (X + Y))).contiguous()
    p = Bd.make_params(n, n, dx, dt, ref.gamma, np.asarray(ref.sigma) / dt, 0, 0, Bd.FP32)
    with Bd.Grid(p, rho, ux, uy, T) as g:
        del rho, ux, uy, T
        assert g.info()["kernel"] == Bd.KERNEL_TMA and g.info()["tile"] == 6
        t0 = g.totals()
        g.step(3)
        f3 = torch.empty((16, n, n), dtype=torch.float32, device="cuda")
        g.get_f(out=f3)
        g.step(1)
        assert g.health() == Bd.MRT_OK
        t4 = g.totals()
        rng = np.random.default_rng(16384)
        m = 48
        wins = [(0, 0), (n - m, n - m), (0, n - m), (n - m, 0), (5000, 128 * 40 - 24)]
        wins += [(int(rng.integers(0, n - m)), int(rng.integers(0, n - m))) for _ in range(7)]
        got, src = [], []
        for (y0, x0) in wins:
            ys = torch.arange(y0 - 1, y0 + m + 1, device="cuda") % n
            xs = torch.arange(x0 - 1, x0 + m + 1, device="cuda") % n
            src.append(f3[:, ys][:, :, xs].double().cpu().numpy())
        del f3
        f4 = torch.empty((16, n, n), dtype=torch.float32, device="cuda")
        g.get_f(out=f4)
        for (y0, x0) in wins:
            got.append(f4[:, y0:y0 + m, x0:x0 + m].double().cpu().numpy())
        del f4
    b = 2.0 / (ref.gamma - 1.0)
    for (y0, x0), fw, fg in zip(wins, src, got):
        og = oracle.Grid(m + 2, m + 2, dx, dt, b, np.asarray(p.s[:]), oracle.BC_PERIODIC, oracle.BC_PERIODIC)
        og.gx = np.zeros((16, 2, m + 2))
        og.gy = np.zeros((16, 2, m + 2))
        want = oracle.step(og, np.ascontiguousarray(fw))[:, 1:-1, 1:-1]
        assert np.max(np.abs(fg - want)) <= 2e-6 * np.max(np.abs(want)), (y0, x0)
    # mass and energy are conserved; FP32 state rounding over 4 steps of 268 M cells
    np.testing.assert_allclose(t4[[0, 3]], t0[[0, 3]], rtol=1e-6)
