"""Open channels on the GPU (column pass + masked tiles) against the FP64
oracle: an Oldroyd-B channel with a mismatched inlet profile, and the
paper's cylinder set-up (inlet profile, outlet at density 1, curved walls)
at the oracle size R = 8; FP32, tile-width independence, checkpoint /
resume and the host-side rejections.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from gpu_helpers import parity_errors
from oracle_helpers import oracle_sim
from paper_2508_16997_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def lbve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16997_gb300 import build, lbve as L
    build.build()
    return L


def open_channel():
    """Walled Oldroyd-B channel, open in x, body-force driven, with an inlet
    profile that does not match the channel's own steady state (a
    transverse inlet velocity included)."""
    H, nx = 14, 23
    inst = wl.channel(H, nx=nx, Wi=2.0, Sc=1e3)
    Uc = wl.velocity_scale(inst.Ma)
    prof = wl.poiseuille_inlet(H, 1.4 * Uc, 30.0)
    prof[1] = 0.1 * prof[0]
    inst.open_x = True
    inst.inlet = prof
    return inst


CASES = {
    "open_channel": open_channel,
    "cylinder_open_r8": lambda: wl.cylinder_channel(8, open_x=True),
}


def run_pair(L, inst, steps, precision=0, init=None, tile_tx=0):
    sim = L.Simulation([inst], precision=precision,
                       init_fields=None if init is None else [init], tile_tx=tile_tx)
    o = oracle_sim(inst, init=init)
    if inst.solid is not None:
        o.set_mask(inst.solid, inst.wall_q)
    sim.step(steps)
    o.step(steps)
    return sim, o


@pytest.mark.parametrize("case", sorted(CASES))
def test_open_fp64_parity(lbve, case):
    inst = CASES[case]()
    init = wl.random_fields(inst.nx, inst.ny, seed=51)
    sim, o = run_pair(lbve, inst, 150, init=init)
    g, r = sim.fields(0), o.fields()
    err = parity_errors(g, r)
    assert err["u"] <= FP64_TOL and err["C"] <= FP64_TOL and err["C-I"] <= 100 * FP64_TOL, err
    assert np.abs(g[0] - r[0]).max() <= 1e-13
    tg, to = sim.totals(0), o.totals()
    np.testing.assert_allclose(tg[:6], to[:6], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(tg[6:14], to[6:14], rtol=1e-9, atol=1e-13)


def test_open_cylinder_fp32(lbve):
    inst = CASES["cylinder_open_r8"]()
    sim, o = run_pair(lbve, inst, 300, precision=1)
    err = parity_errors(sim.fields(0), o.fields())
    assert err["u"] <= FP32_TOL and err["C"] <= FP32_TOL, err


@pytest.mark.parametrize("precision", [0, 1])
def test_open_tile_width_independent(lbve, precision):
    inst = open_channel()
    ref = lbve.Simulation([inst], precision=precision)
    ref.step(60)
    for tx in (1, 5, 8, 16):
        s = lbve.Simulation([inst], precision=precision, tile_tx=tx)
        s.step(60)
        np.testing.assert_array_equal(s.fields(0), ref.fields(0), err_msg=f"tile_tx={tx}")


def test_open_mixed_batch(lbve):
    """Open, masked and periodic instances of both precisions in one handle
    run as they do alone."""
    mk = [open_channel, lambda: wl.frm(20, Wi=1.0, Re=1.0, Ma=0.05), CASES["cylinder_open_r8"],
          lambda: wl.channel(10, nx=5, Wi=2.0)]
    precs = [0, 1, 0, 1]
    batch = lbve.Simulation([f() for f in mk], precision=precs)
    batch.step(41)
    for i, (f, p) in enumerate(zip(mk, precs)):
        alone = lbve.Simulation([f()], precision=p)
        alone.step(41)
        np.testing.assert_array_equal(batch.fields(i), alone.fields(0), err_msg=str(i))


def test_open_save_load_and_rejections(lbve):
    L = lbve
    inst = open_channel()
    a = L.Simulation([inst], precision=0)
    a.step(25)
    state = L.lbve_save(a.h)
    a.step(30)
    b = L.Simulation([inst], precision=0)
    L.lbve_load(b.h, state)
    b.step(30)
    np.testing.assert_array_equal(a.fields(0), b.fields(0))
    other = open_channel()
    other.inlet = other.inlet * 1.01
    c = L.Simulation([other], precision=0)
    with pytest.raises(L.LbveError) as e:
        L.lbve_load(c.h, state)
    assert e.value.code == L.LBVE_ERR_GEOMETRY
    # the inlet of a periodic instance; the adjoint of an open channel with
    # a zero loss (its gradients are test_gpu_adjoint_open.py's)
    per = L.Simulation([wl.channel(8, nx=6)])
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_inlet(per.h, 0, np.zeros((5, 9)))
    assert e.value.code == L.LBVE_ERR_GEOMETRY
    import torch
    g = torch.zeros((6, inst.ny, inst.nx), dtype=torch.float64, device="cuda")
    dF = torch.zeros((2, inst.ny, inst.nx), dtype=torch.float64, device="cuda")
    nb = L.lbve_adjoint_workspace_bytes(a.h, 0, 4)
    aws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    dF.fill_(1.0)
    L.lbve_adjoint_step(a.h, 0, None, g.data_ptr(), 4, aws.data_ptr(), nb, dF.data_ptr(),
                        inst.n_nodes)
    assert bool((dF == 0).all())
    # a mask too close to an open column
    bad = open_channel()
    m = np.zeros((bad.ny, bad.nx), np.uint8)
    m[7, 2] = 1
    bad.solid = m
    with pytest.raises(L.LbveError) as e:
        L.Simulation([bad])
    assert e.value.code == L.LBVE_ERR_GEOMETRY
