"""Steady drag on a cylinder in a channel (Sec. 4.3), for comparison with the
paper's printed drag coefficients.

Set-up of Sec. 4.3: a 30R x 4R channel (wet-node walls on rows 0 and 4R),
the cylinder at (15R, 2R), an inlet column carrying the fully developed
Oldroyd-B channel profile with mean velocity U_c (U_max = 1.5 U_c), an outlet
column at density 1; Re = 1, beta = 0.59, Sc = 1e6, Lambda_p = 2.5e-7,
Lambda_s = 1/4, Ma = 0.01, L_c = R.  The cylinder wall uses CNEBB for the
conformation lattices and interpolated bounce-back at the exact circle link
fractions for the hydrodynamic lattice.

All (R, Wi) cases advance together in one batch, in chunks of one
convective time R/U_c (t* = 1 per chunk, chunk length of the largest R),
until each case's residual max|u(t) - u(t - chunk)|/U_c is below ``tol``,
or until the wall-clock budget runs out.  Printed per case, one JSON line:
C_d = F_x / (1/2 rho U_c^2 2R) from the momentum-exchange force on the
cylinder, steps, residual, and the paper's value for the CNEBB scheme
(its drag table at Sc = 1e6).

    python -m paper_2508_16997_gb300.cylinder_drag --R 10,20,40 --Wi 0.1,0.5,1.0
"""
import argparse
import json
import time

from . import lbve as L
from . import workloads as wl

# The paper's steady drag coefficients, CNEBB column of its table for
# Sc = 1e6 (Sec. 4.3), keyed by (R, Wi).
PAPER_CD = {
    (5, 0.1): 106.93, (5, 0.5): 103.88,
    (10, 0.1): 125.90, (10, 0.5): 121.26, (10, 1.0): 165.30,
    (15, 0.1): 128.52, (15, 0.5): 123.21, (15, 1.0): 161.91,
    (20, 0.1): 129.59, (20, 0.5): 124.84, (20, 1.0): 158.44,
    (25, 0.1): 129.69, (25, 0.5): 124.60, (25, 1.0): 152.98,
    (30, 0.1): 130.42, (30, 0.5): 125.88, (30, 1.0): 147.14,
    (35, 0.1): 130.83, (35, 0.5): 127.30, (35, 1.0): 143.66,
    (40, 0.1): 130.83, (40, 0.5): 126.39, (40, 1.0): 140.32,
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--R", default="10,20,40")
    ap.add_argument("--Wi", default="0.1,0.5,1.0")
    ap.add_argument("--precision", type=int, default=L.LBVE_FP64)
    ap.add_argument("--tol", type=float, default=1e-7)
    ap.add_argument("--budget-s", type=float, default=900.0)
    a = ap.parse_args(argv)
    cases = [(int(r), float(w)) for r in a.R.split(",") for w in a.Wi.split(",")]
    insts = [wl.cylinder_channel(r, Wi=w, open_x=True) for r, w in cases]
    Uc = wl.velocity_scale(insts[0].Ma)
    chunk = int(round(max(r for r, _ in cases) / Uc))
    sim = L.Simulation(insts, precision=a.precision)
    t0 = time.time()
    steps, done = 0, [None] * len(cases)
    while any(d is None for d in done) and time.time() - t0 < a.budget_s:
        sim.step(chunk)
        steps += chunk
        flags = sim.status()
        for i in range(len(cases)):
            if done[i] is None and (flags[i] or sim.residual(i) < a.tol):
                done[i] = steps
        if flags.all():
            break
    flags = sim.status()
    for i, (r, w) in enumerate(cases):
        tot = sim.totals(i)
        cd = tot[12] / (Uc * Uc * r)
        print(json.dumps(dict(R=r, Wi=w, precision=a.precision, steps=steps, t_star=steps * Uc / r,
                              converged_at=done[i], residual=sim.residual(i),
                              nonfinite=bool(flags[i]), Cd=cd, paper_Cd=PAPER_CD.get((r, w)),
                              rel_diff=(cd / PAPER_CD[(r, w)] - 1.0)
                              if (r, w) in PAPER_CD else None)), flush=True)
    print(json.dumps(dict(seconds=time.time() - t0, steps=steps)), flush=True)


if __name__ == "__main__":
    main()
