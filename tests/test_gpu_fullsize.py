"""Parity at full size, in the launch configuration the benchmark times.

The benchmark advances the 256-instance batched mix (128 Oldroyd-B channels
with H ~ U{32..512}, nx = 4, and 128 four-roll mills with N ~ U{64..512}) in
float32-deviation storage, one launch per step, with CUDA-graph replays of
32-step runs.  This test runs exactly that handle for 40 steps (one replay,
seven single steps, the final step) and checks sampled outputs against the
float64 oracle:

  * channels are small enough (at most 4 x 513 nodes) for the oracle to run
    whole: three of them are compared on every node;
  * a four-roll mill of N^2 up to 512^2 nodes is compared on 9 x 9 patches.
    After T steps a node depends only on nodes within 2T + 1 of it (each step
    pulls from the nearest neighbours and takes gradients of their moments;
    the initial collision adds one more ring), so the oracle run on the
    periodic window of half-width 90 around a patch -- same parameters, the
    window's slice of the force field, the same rest initial state --
    reproduces the patch exactly for T = 40 (90 >= 2 T + 1 + 4 + 1); its own
    wrap-around only disturbs nodes outside the dependency cone.

Tolerance: relative L2 <= 1e-5 on u and on C (the float32 target), and the
density within 1e-6.  Every instance of the mix must stay finite, and the
total mass of every four-roll mill (a periodic box) must stay N^2 to 1e-12
relative."""
import numpy as np
import pytest

import bench
from gpu_helpers import rel_l2
from oracle_helpers import oracle_sim
from paper_2508_16997_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STEPS = 40
HALF = 90   # window half-width: >= 2 STEPS + 1 + patch radius + 1
PATCH = 4   # patch radius (9 x 9 patch)
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def lbve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16997_gb300 import build, lbve as L
    build.build()
    return L


@pytest.fixture(scope="module")
def full_mix(lbve):
    insts = bench.workload(0, bench.N_INSTANCES)
    sim = lbve.Simulation(insts, precision=lbve.LBVE_FP32_DEV)
    sim.step(STEPS)
    return insts, sim


def _window(inst, cx, cy, h):
    """The instance restricted to the periodic window of half-width h
    centred at (cx, cy): same parameters, the window's force field."""
    N = inst.nx
    xs = np.arange(cx - h, cx + h + 1) % N
    ys = np.arange(cy - h, cy + h + 1) % N
    F = inst.force_field[:, ys][:, :, xs]
    return wl.Instance(2 * h + 1, 2 * h + 1, True, inst.beta, inst.Wi, inst.Re, inst.Sc,
                       inst.Ma, inst.Lc, inst.Lambda_s, inst.Lambda_p, 0.0, 0.0, "window",
                       np.ascontiguousarray(F), inst.seed)


def _compare(got, ref, what):
    eu, eC = rel_l2(got[1:3], ref[1:3]), rel_l2(got[3:6], ref[3:6])
    drho = float(np.abs(got[0] - ref[0]).max())
    assert eu <= FP32_TOL and eC <= FP32_TOL and drho <= 1e-6, (what, eu, eC, drho)


def test_full_mix_channels_every_node(full_mix):
    insts, sim = full_mix
    ch = [i for i, x in enumerate(insts) if x.kind == "channel"]
    by_h = sorted(ch, key=lambda i: insts[i].ny)
    for i in (by_h[0], by_h[len(by_h) // 2], by_h[-1]):
        o = oracle_sim(insts[i])
        o.step(STEPS)
        _compare(sim.fields(i), o.fields(), f"channel {i} ({insts[i].nx} x {insts[i].ny})")


def test_full_mix_four_roll_mill_patches(full_mix):
    insts, sim = full_mix
    frm = [i for i, x in enumerate(insts) if x.kind == "frm"]
    rng = np.random.default_rng(2025)
    largest = max(frm, key=lambda i: insts[i].nx)
    picks = [largest] + [int(i) for i in rng.choice(frm, 2, replace=False) if i != largest][:2]
    checked = 0
    for i in picks:
        inst = insts[i]
        N = inst.nx
        got_all = sim.fields(i)
        if N <= 2 * HALF + 1:  # small enough to run whole
            o = oracle_sim(inst)
            o.step(STEPS)
            _compare(got_all, o.fields(), f"frm {i} (N = {N}) whole")
            checked += 1
            continue
        for cx, cy in rng.integers(0, N, size=(2, 2)):
            w = _window(inst, int(cx), int(cy), HALF)
            o = oracle_sim(w)
            o.step(STEPS)
            ref = o.fields()[:, HALF - PATCH:HALF + PATCH + 1, HALF - PATCH:HALF + PATCH + 1]
            xs = np.arange(cx - PATCH, cx + PATCH + 1) % N
            ys = np.arange(cy - PATCH, cy + PATCH + 1) % N
            got = got_all[:, ys][:, :, xs]
            _compare(got, ref, f"frm {i} (N = {N}) patch at ({cx}, {cy})")
            checked += 1
    assert checked >= 3


def test_full_mix_invariants(full_mix):
    insts, sim = full_mix
    assert not sim.status().any()
    for i, inst in enumerate(insts):
        if inst.kind != "frm":
            continue
        mass = sim.totals(i)[0]
        n = inst.nx * inst.ny
        assert abs(mass - n) <= 1e-12 * n, (i, mass, n)


@pytest.mark.parametrize("precision", [0, 1])
def test_maximum_grid_patches(lbve, precision):
    """The largest grid a handle takes, 8192 x 4096 = 2^25 nodes (36 planes of
    indices just inside int32), periodic, with a random per-node force: after
    10 steps, 9 x 9 patches at the start, the middle and the very end of the
    arrays match the oracle on their periodic windows (half-width 30 >=
    2 T + 1 + 4 + 1).  Float64 to 1e-12, float32 to 1e-5.  The force
    amplitude 1e-3 keeps u near 1e-3: the oracle stores full populations
    (about 0.1), whose round-off leaves about 1e-16 absolute in u, so with a
    1e-5 force (u near 1e-5) the two sides differed by 1e-11 relative on any
    grid size, 256 x 128 included."""
    nx, ny, T, h = 8192, 4096, 10, 30
    inst = wl.Instance(nx, ny, True, 0.5, 2.0, 1.0, 1e4, 0.1, ny / (2 * np.pi), 0.25, 1e-6,
                       kind="custom")
    inst.force_field = wl.random_force(nx, ny, seed=77, amp=1e-3)
    sim = lbve.Simulation([inst], precision=precision)
    sim.step(T)
    assert not sim.status().any()
    got_all = sim.fields(0)
    tol = 1e-12 if precision == 0 else FP32_TOL
    for cx, cy in ((2, 1), (nx // 2 + 17, ny // 2 - 5), (nx - 3, ny - 2)):
        xs = np.arange(cx - h, cx + h + 1) % nx
        ys = np.arange(cy - h, cy + h + 1) % ny
        F = inst.force_field[:, ys][:, :, xs]
        w = wl.Instance(2 * h + 1, 2 * h + 1, True, inst.beta, inst.Wi, inst.Re, inst.Sc, inst.Ma,
                        inst.Lc, inst.Lambda_s, inst.Lambda_p, 0.0, 0.0, "window",
                        np.ascontiguousarray(F))
        o = oracle_sim(w)
        o.step(T)
        ref = o.fields()[:, h - PATCH:h + PATCH + 1, h - PATCH:h + PATCH + 1]
        pxs = np.arange(cx - PATCH, cx + PATCH + 1) % nx
        pys = np.arange(cy - PATCH, cy + PATCH + 1) % ny
        got = got_all[:, pys][:, :, pxs]
        eu, eC = rel_l2(got[1:3], ref[1:3]), rel_l2(got[3:6], ref[3:6])
        assert eu <= tol and eC <= tol, (precision, cx, cy, eu, eC)
    del sim
