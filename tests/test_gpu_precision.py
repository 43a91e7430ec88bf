"""FP32 drift over a long run: the Kelvin-Helmholtz shear layer at 1024^2
for 5000 steps (the step count of the 4096^2 configuration).  FP32 keeps
the bulk state and every step of the update, including the closure
T = (e - j^2/rho)/(b rho) and the equilibrium moments; FP64 is used only to
accumulate the conserved totals.  This test is what keeps it that way: the
FP32 run must stay within 1e-5 (L-inf and L1, relative) of the FP64 run in
rho, u, v and T, and its conserved totals within 1e-5 of their starting
values (relative to the sum of |q| per quantity)."""
import numpy as np
import pytest

import oracle
from paper_1004_5442_gb300 import binding as Bd
from paper_1004_5442_gb300 import workloads as W
from _parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    Bd.load()
    yield


def test_fp32_drift_5000_steps():
    w = W.kelvin_helmholtz(n=1024, nsteps=5000)
    with Bd.Grid.from_workload(w, precision=Bd.FP64) as g64:
        f0 = g64.get_f()
        g64.step(w.nsteps)
        want = g64.macro()
        t64 = g64.totals()
    _, _, _, M, _ = oracle.model()
    absq = np.array([np.sum(np.abs(np.tensordot(M[k], f0, 1))) * w.dx ** 2 for k in range(4)])
    with Bd.Grid.from_workload(w, precision=Bd.FP32) as g32:
        g32.step(1)
        start = g32.totals()
        g32.step(w.nsteps - 1)
        got = g32.macro()
        t32 = g32.totals()
    errs = assert_parity(got, want, linf=1e-5, l1=1e-5, label="fp32 vs fp64, 5000 steps")
    drift = np.abs(t32 - start) / absq
    print("fp32 vs fp64", errs, "fp32 totals drift", drift, "fp64 vs fp32 totals", np.abs(t64 - t32) / absq)
    assert np.all(drift <= 1e-5)
    assert np.all(np.abs(t64 - t32) <= 1e-5 * absq)
