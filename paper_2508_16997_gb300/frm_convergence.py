"""Grid convergence of the four-roll mill (Sec. 4.1), in the form the paper
reports it: steady u_x, u_y, A_xx, A_xy, A_yy at the 33 x 33 monitoring
points spaced pi/16, compared with the finest grid by the root-mean-square
error E = sqrt(mean_k (q(x_k) - q_ref(x_k))^2), and the slope of log E
against log N fitted by least squares (with R^2) over the grids named by
``--fit``.

Set-up of the section: N unique periodic nodes per axis, Re = 1,
beta = 2/3, Sc = 1e5, Ma = 0.01, Lambda_s = 1/4, Lambda_p = 1e-6, the
forcing F0 = 2 mu_s U_c (2 pi / N)^2, started from the Newtonian steady
field with A = I and run for ``--tstar`` convective times L_c / U_c.
The paper uses N = 32 ... 2048 with N = 2048 as the reference and fits
N = 128 ... 2048; the default here is one level coarser (reference 1024).

    python -m paper_2508_16997_gb300.frm_convergence --N 64,128,256,512,1024 --Wi 5

``--save`` keeps the monitor values (one (5, 33, 33) array per N) for
further comparison, e.g. of two run lengths.
"""
import argparse
import json
import math
import time

import numpy as np

from . import lbve as L
from . import workloads as wl

FIELDS = ("ux", "uy", "Axx", "Axy", "Ayy")


def monitor(f: np.ndarray, N: int) -> np.ndarray:
    """The five fields at the 33 x 33 points x~ = k pi/16 (node k N/32, the
    last row and column wrapping onto the first)."""
    idx = (np.arange(33) * N // 32) % N
    return np.stack([f[c][np.ix_(idx, idx)] for c in (1, 2, 3, 4, 5)])


def run(N: int, Wi: float, tstar: float, precision: int):
    inst = wl.frm(N, beta=2.0 / 3.0, Wi=Wi, Re=1.0, Ma=0.01, Sc=1e5, Lambda_s=0.25,
                  Lambda_p=1e-6, force_visc="nus")
    Uc = wl.velocity_scale(inst.Ma)
    Tc = inst.Lc / Uc
    xt = 2 * math.pi * np.arange(N) / N
    X, Y = np.meshgrid(xt, xt, indexing="xy")
    init = np.zeros((6, N, N))
    init[0] = init[3] = init[5] = 1.0
    init[1] = Uc * np.sin(X) * np.cos(Y)
    init[2] = -Uc * np.cos(X) * np.sin(Y)
    sim = L.Simulation([inst], precision=precision, init_fields=[init])
    steps = int(round(tstar * Tc))
    t0 = time.time()
    sim.step(steps)
    f = sim.fields(0)
    return monitor(f, N), steps, time.time() - t0, bool(sim.status()[0]), Uc


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--N", default="64,128,256,512,1024")
    ap.add_argument("--fit", default="128,256,512")
    ap.add_argument("--Wi", type=float, default=5.0)
    ap.add_argument("--tstar", type=float, default=60.0)
    ap.add_argument("--precision", type=int, default=L.LBVE_FP32_DEV)
    ap.add_argument("--save", default="", help="write the monitor values per N to this .npz")
    a = ap.parse_args(argv)
    Ns = sorted(int(n) for n in a.N.split(","))
    res = {}
    for N in Ns:
        m, steps, secs, bad, Uc = run(N, a.Wi, a.tstar, a.precision)
        res[N] = m
        print(json.dumps(dict(N=N, steps=steps, seconds=secs, nonfinite=bad)), flush=True)
    if a.save:
        np.savez(a.save, **{f"N{N}": res[N] for N in Ns}, Wi=a.Wi, tstar=a.tstar)
    ref = res[Ns[-1]]
    errs = {N: np.sqrt(((res[N] - ref) ** 2).reshape(5, -1).mean(axis=1)) for N in Ns[:-1]}
    for N in Ns[:-1]:
        print(json.dumps(dict(N=N, **{k: float(v) for k, v in zip(FIELDS, errs[N])},
                              ux_over_Uc=float(errs[N][0] / Uc))), flush=True)
    fit = [N for N in (int(n) for n in a.fit.split(",")) if N in errs]
    if len(fit) < 2:
        return
    lx = np.log(np.array(fit, dtype=float))
    for c, name in enumerate(FIELDS):
        ly = np.log(np.array([errs[N][c] for N in fit]))
        slope, icpt = np.polyfit(lx, ly, 1)
        pred = slope * lx + icpt
        r2 = 1.0 - ((ly - pred) ** 2).sum() / ((ly - ly.mean()) ** 2).sum()
        print(json.dumps(dict(field=name, order=-float(slope), R2=float(r2), fit=fit,
                              reference=Ns[-1], Wi=a.Wi)), flush=True)


if __name__ == "__main__":
    main()
