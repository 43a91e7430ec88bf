"""Expected values of the reverse-mode configuration: gradient of
L = 1/2 sum (rho_N - rho_target)^2 dx^2 after 500 steps of the 512 x 512
periodic smooth vortex (Ma 0.8, gamma 1.4, Pr 0.71, sigma 0.05, checkpoints
every 50 steps), with respect to the initial (rho, u_x, u_y, T) fields and
the 16 relaxation rates, from the FP64 oracle's reverse mode; and central
differences of the oracle's loss (h = 1e-4: absolute along seeded field
directions, relative for five rates).

The oracle's reverse sweep is serial (about 4 minutes here for 500 steps of
512^2), too slow to run inside a test, so the values are stored in
vortex_adjoint_512.json beside this script:
  * the loss and the 16 rate gradients;
  * per field, the L2 norm of its gradient, its value at 2048 seeded cells
    and its dot product with four seeded standard-normal directions;
  * the central differences of the loss along the first direction of each
    field and along s_5, s_6, s_8, s_10 and s_14 (s_k (1 +- h)).
The directions come from numpy default_rng(SEED + 10 * field + j) and the
sampled cells from default_rng(SEED), so a test regenerates them.

Calls only oracle/ and the input generator.  Run from the repository root:
    python tests/golden/write_vortex_adjoint.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1004_5442_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "vortex_adjoint_512.json")
SEED = 20100430
N, NSTEPS, CKPT = 512, 500, 50
H = 1e-4
FIELDS = ("rho", "ux", "uy", "T")
RATES = (4, 5, 7, 9, 13)      # 0-based: s_5, s_6, s_8, s_10, s_14
NSAMPLE = 2048
NDIR = 4


def workload():
    w = W.smooth_vortex(n=N, nsteps=NSTEPS)
    return w, W.vortex_target(w)


def loss_grad(target, dx):
    def lg(r):
        d = r - target
        return 0.5 * float(np.sum(d * d)) * dx * dx, d * dx * dx
    return lg


def sample_cells():
    return np.sort(np.random.default_rng(SEED).choice(N * N, NSAMPLE, replace=False))


def direction(field, j):
    return np.random.default_rng(SEED + 10 * field + j).standard_normal((N, N))


def main():
    w, target = workload()
    lg = loss_grad(target, w.dx)
    t0 = time.time()
    L, g_rho, g_ux, g_uy, g_T, g_s = oracle.adjoint_run(w.nx, w.ny, w.dx, w.dt, w.b, w.s, w.rho, w.ux, w.uy,
                                                        w.T, NSTEPS, lg, w.bc_x, w.bc_y, ckpt=CKPT)
    print(f"reverse mode: {time.time() - t0:.0f} s, L = {L!r}", flush=True)
    grads = (g_rho, g_ux, g_uy, g_T)
    cells = sample_cells()
    fields = {}
    base = dict(rho=w.rho, ux=w.ux, uy=w.uy, T=w.T)

    def loss_of(s=None, **kw):
        a = dict(base)
        a.update(kw)
        return oracle.forward_loss(w.nx, w.ny, w.dx, w.dt, w.b, w.s if s is None else s, a["rho"], a["ux"],
                                   a["uy"], a["T"], NSTEPS, lg, w.bc_x, w.bc_y)

    for q, (name, g) in enumerate(zip(FIELDS, grads)):
        dots = [float(np.sum(g * direction(q, j))) for j in range(NDIR)]
        d0 = direction(q, 0)
        t0 = time.time()
        fd = (loss_of(**{name: base[name] + H * d0}) - loss_of(**{name: base[name] - H * d0})) / (2 * H)
        print(f"{name}: dot {dots[0]!r} fd {fd!r} rel {abs(dots[0] - fd) / abs(fd):.2e}"
              f" ({time.time() - t0:.0f} s)", flush=True)
        fields[name] = {"l2": float(np.linalg.norm(g)), "sum_abs": float(np.sum(np.abs(g))),
                        "samples": [float(v) for v in g.ravel()[cells]], "dots": dots, "fd_dir0": float(fd)}
    rates_fd = {}
    for k in RATES:
        sp, sm = w.s.copy(), w.s.copy()
        sp[k] *= 1 + H
        sm[k] *= 1 - H
        fd = (loss_of(s=sp) - loss_of(s=sm)) / (2 * H)
        print(f"s_{k + 1}: s*dL/ds {g_s[k] * w.s[k]!r} fd {fd!r}", flush=True)
        rates_fd[str(k)] = float(fd)
    doc = {"_source": "tests/golden/write_vortex_adjoint.py (FP64 oracle reverse mode and central differences)",
           "n": N, "nsteps": NSTEPS, "ckpt": CKPT, "seed": SEED, "h": H, "nsample": NSAMPLE, "ndir": NDIR,
           "loss": float(L), "g_s": [float(v) for v in g_s], "s": [float(v) for v in w.s],
           "fields": fields, "rates_fd": rates_fd}
    with open(OUT, "w") as fh:
        json.dump(doc, fh)
    print("written", OUT)


if __name__ == "__main__":
    main()
