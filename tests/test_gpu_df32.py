"""LBVE_DF32: storage and arithmetic in float32 pairs (about 48 significant
bits, error-free float32 transformations on the float32 pipe).

Parity with the FP64 oracle on the parity cases of the float64 path, the
fields independent of the tile width, and the long horizons where float32
deviation storage drifts: the Wi-sweep channels against the float64 path after
the 1.06 M steps that Wi = 100 needs to reach its steady state."""
import numpy as np
import pytest

from gpu_helpers import parity_errors
from oracle_helpers import oracle_sim
from paper_2508_16997_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DF_TOL = 1e-10


@pytest.fixture(scope="module")
def lbve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16997_gb300 import build, lbve as L
    build.build()
    return L


def _rel(a, r):
    return (float(np.linalg.norm(a[1:3] - r[1:3]) / np.linalg.norm(r[1:3])),
            float(np.linalg.norm(a[3:6] - r[3:6]) / np.linalg.norm(r[3:6])))


@pytest.mark.parametrize("case", ["frm64", "channel", "ragged"])
def test_df32_parity_with_the_oracle(lbve, case):
    """Against the FP64 oracle, relative L2 of u, C and C - I within 1e-10:
    the four-roll mill 64^2 as specified (2000 steps), the walled channel
    (H = 16, Wi = 10, 1500 steps), and a ragged random-state periodic grid
    with a random force field (37 x 21, 150 steps)."""
    if case == "frm64":
        inst, steps, init = wl.frm(64), 2000, None
    elif case == "channel":
        inst, steps, init = wl.channel(16, nx=4, Wi=10.0), 1500, None
    else:
        inst = wl.Instance(37, 21, True, 0.6, 0.8, 1.0, 1e3, 0.1, 37 / (2 * np.pi), 0.25, 1e-4,
                           0.0, 0.0, "custom")
        inst.force_field = wl.random_force(37, 21, seed=3, amp=1e-5)
        steps, init = 150, wl.random_fields(37, 21, seed=4)
    sim = lbve.Simulation([inst], precision=lbve.LBVE_DF32,
                          init_fields=None if init is None else [init])
    sim.step(steps)
    o = oracle_sim(inst, init=init)
    o.step(steps)
    e = parity_errors(sim.fields(0), o.fields())
    assert e["u"] <= DF_TOL and e["C"] <= DF_TOL and e["C-I"] <= 100 * DF_TOL, (case, e)
    assert not sim.status().any()


def test_df32_tile_width_does_not_change_fields(lbve):
    insts = [wl.frm(40, Wi=2.0, Re=1.0, Ma=0.05), wl.channel(20, nx=4, Wi=30.0)]
    inits = [wl.random_fields(i.nx, i.ny, seed=11 + k) for k, i in enumerate(insts)]
    ref = lbve.Simulation(insts, precision=lbve.LBVE_DF32, init_fields=inits)
    ref.step(40)
    for tx in (1, 8, 16):
        widths = [min(tx, i.nx) for i in insts]
        s = lbve.Simulation(insts, precision=lbve.LBVE_DF32, init_fields=inits, tile_tx=widths)
        s.step(40)
        for i in range(len(insts)):
            np.testing.assert_array_equal(s.fields(i), ref.fields(i))


def test_df32_channels_keep_float64_accuracy_over_long_horizons(lbve):
    """The three Wi-sweep channels (H = 64, Wi = 1, 10, 100) after 1,059,095
    steps, the number Wi = 100 needs to reach its steady state: LBVE_DF32
    against the float64 path within 1e-8 in u and C (float32 deviation
    storage drifts by 4e-6..9e-5 over such horizons)."""
    insts = [wl.channel(64, nx=4, Wi=w) for w in (1.0, 10.0, 100.0)]
    d = lbve.Simulation(insts, precision=lbve.LBVE_DF32)
    f = lbve.Simulation(insts, precision=lbve.LBVE_FP64)
    d.step(1059095)
    f.step(1059095)
    for i, inst in enumerate(insts):
        eu, eC = _rel(d.fields(i), f.fields(i))
        assert eu <= 1e-8 and eC <= 1e-8, (inst.Wi, eu, eC)


def test_df32_rejects_what_it_does_not_cover(lbve):
    bad = lbve.params_from(wl.cylinder_channel(8), lbve.LBVE_DF32)
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_workspace_bytes([bad])
    assert e.value.code == lbve.LBVE_ERR_ARG
