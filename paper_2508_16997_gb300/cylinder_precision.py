"""Flow past a cylinder at R = 64 (Sec. 4.3 set-up), FP32 against FP64.

The channel is 30R x 4R (1920 x 257 nodes, wet-node walls on rows 0 and
4R), with the cylinder at (15R, 2R), the fully developed Oldroyd-B inlet
profile with mean U_c, an outlet column at density 1, Re = 1, beta = 0.59,
Sc = 1e6, Lambda_p = 2.5e-7, Ma = 0.01 and curved-wall link fractions of
the exact circle.  Every Wi runs in float64 and in float32-deviation storage
for the same number of steps, starting from rest.  Printed per Wi, one JSON
line:
  - the drag coefficient C_d = F_x / (1/2 rho U_c^2 2R) in both precisions
    (momentum exchange on the cylinder) and their relative difference;
  - the relative L2 difference of A_xx along the wake centreline (row 2R,
    from the cylinder's rear x = 16R to the outlet);
  - the MLUPS of each batch (fluid nodes x steps / time).

    python -m paper_2508_16997_gb300.cylinder_precision --Wi 0.1,0.5 --steps 200000
"""
import argparse
import json
import time

import numpy as np

from . import lbve as L
from . import workloads as wl


def run(insts, precision, steps, chunk):
    import torch
    sim = L.Simulation(insts, precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        n = min(chunk, steps - done)
        sim.step(n)
        done += n
    torch.cuda.synchronize()
    return sim, time.perf_counter() - t0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--R", type=int, default=64)
    ap.add_argument("--Wi", default="0.1,0.5,1.0")
    ap.add_argument("--steps", type=int, default=200000)
    a = ap.parse_args(argv)
    R = a.R
    Wis = [float(w) for w in a.Wi.split(",")]
    insts = [wl.cylinder_channel(R, Wi=w, open_x=True) for w in Wis]
    Uc = wl.velocity_scale(insts[0].Ma)
    fluid = sum(int((i.solid == 0).sum()) for i in insts)
    out = {}
    for prec, tag in ((L.LBVE_FP64, "fp64"), (L.LBVE_FP32_DEV, "fp32")):
        sim, secs = run(insts, prec, a.steps, 20000)
        flags = sim.status()
        out[tag] = dict(seconds=secs, MLUPS=fluid * a.steps / secs / 1e6,
                        cd=[float(sim.totals(i)[12] / (Uc * Uc * R)) for i in range(len(Wis))],
                        axx=[sim.fields(i)[3][2 * R, 16 * R:].copy() for i in range(len(Wis))],
                        finite=[not bool(f) for f in flags])
        del sim
    for i, w in enumerate(Wis):
        c64, c32 = out["fp64"]["cd"][i], out["fp32"]["cd"][i]
        a64, a32 = out["fp64"]["axx"][i], out["fp32"]["axx"][i]
        print(json.dumps(dict(R=R, Wi=w, steps=a.steps, t_star=a.steps * Uc / R,
                              Cd_fp64=c64, Cd_fp32=c32, Cd_rel_diff=c32 / c64 - 1.0,
                              wake_Axx_rel_l2=float(np.linalg.norm(a32 - a64) /
                                                    np.linalg.norm(a64)),
                              wake_Axx_max_fp64=float(a64.max()),
                              finite=[out["fp64"]["finite"][i], out["fp32"]["finite"][i]])),
              flush=True)
    print(json.dumps(dict(MLUPS_fp64=out["fp64"]["MLUPS"], MLUPS_fp32=out["fp32"]["MLUPS"],
                          seconds_fp64=out["fp64"]["seconds"],
                          seconds_fp32=out["fp32"]["seconds"])), flush=True)


if __name__ == "__main__":
    main()
