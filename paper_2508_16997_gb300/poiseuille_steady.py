"""Oldroyd-B Poiseuille channels run to steady state (Sec. 4.2), FP64 and FP32.

The five channels (one per Wi) advance together in one batch.  The float64
batch steps in chunks of one convective time H/U_c until every instance's
residual max|u(t) - u(t - chunk)|/U_c (eq. 2eq4 form) is below ``tol``, or
until the wall-clock budget runs out.  The float32-deviation batch then runs
the same number of steps in one call.  Each result is printed as one JSON
line:
  - steps to convergence;
  - the global relative error (GRE, sum |num - ana| / sum |ana|) of u_x,
    A_xx - 1 and A_xy against the steady closed form (eq_ux_ana,
    eq_Tab_ana);
  - the FP32 vs FP64 relative L2 of u and of C.

    python -m paper_2508_16997_gb300.poiseuille_steady --H 64 --budget-s 600
"""
import argparse
import json
import math
import time

import numpy as np

from . import lbve as L
from . import workloads as wl


def closed_form(H: int, Wi: float, Uc: float):
    """Steady plane Poiseuille profile on rows y = 0..H: u = U_c 4y*(1-y*),
    A_xy = Wi du*/dy*, A_xx = 1 + 2 (Wi du*/dy*)^2 (Kramers relation with
    lambda = Wi H / U_c)."""
    ys = np.arange(H + 1) / H
    du = 4.0 - 8.0 * ys
    return Uc * 4.0 * ys * (1.0 - ys), 1.0 + 2.0 * (Wi * du) ** 2, Wi * du


def gre(num, ana):
    return float(np.abs(num - ana).sum() / np.abs(ana).sum())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--H", type=int, default=64)
    ap.add_argument("--Wi", default="1,10,100,1000,10000")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--max-steps", type=float, default=2e8)
    ap.add_argument("--budget-s", type=float, default=900.0)
    a = ap.parse_args(argv)
    import torch

    Wis = [float(w) for w in a.Wi.split(",")]
    insts = [wl.channel(a.H, nx=4, beta=0.5, Wi=Wi) for Wi in Wis]
    Uc = wl.velocity_scale(insts[0].Ma)
    chunk = int(round(a.H / Uc))

    def report(sim, tag, steps, conv):
        for i, Wi in enumerate(Wis):
            f = sim.fields(i)
            ue, Axx, Axy = closed_form(a.H, Wi, Uc)
            print(json.dumps(dict(prec=tag, Wi=Wi, steps=steps, converged=conv[i],
                                  gre_u=gre(f[1][:, 0], ue), gre_Axx=gre(f[3][:, 0] - 1, Axx - 1),
                                  gre_Axy=gre(f[4][:, 0], Axy))), flush=True)

    s64 = L.Simulation(insts, precision=L.LBVE_FP64)
    t0 = time.time()
    steps, conv_step = 0, [None] * len(Wis)
    while (steps < a.max_steps and any(c is None for c in conv_step)
           and time.time() - t0 < a.budget_s):
        s64.step(chunk)
        steps += chunk
        for i in range(len(Wis)):
            if conv_step[i] is None and s64.residual(i) < a.tol:
                conv_step[i] = steps
    print(json.dumps(dict(phase="fp64", steps=steps, seconds=time.time() - t0,
                          conv_step=conv_step)), flush=True)
    report(s64, "fp64", steps, [c is not None for c in conv_step])

    s32 = L.Simulation(insts, precision=L.LBVE_FP32_DEV)
    t1 = time.time()
    s32.step(steps)
    torch.cuda.synchronize()
    print(json.dumps(dict(phase="fp32", steps=steps, seconds=time.time() - t1)), flush=True)
    report(s32, "fp32", steps, [False] * len(Wis))
    for i, Wi in enumerate(Wis):
        x, y = s32.fields(i), s64.fields(i)
        print(json.dumps(dict(Wi=Wi, fp32_vs_fp64_u=float(np.linalg.norm(x[1:3] - y[1:3])
                                                        / np.linalg.norm(y[1:3])),
                              fp32_vs_fp64_C=float(np.linalg.norm(x[3:6] - y[3:6])
                                                   / np.linalg.norm(y[3:6])))), flush=True)


if __name__ == "__main__":
    main()
