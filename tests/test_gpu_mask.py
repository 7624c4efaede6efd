"""Solid masks on the GPU (wall pass + masked tiles) against the FP64 oracle.

Cases cover staircase (q = 1/2) and curved (circle link fractions) walls, a
flat-walled channel with a cylinder, two-node gaps that select the
first-order one-sided differences, a mixed batch of masked and unmasked
instances in both precisions, the force on the solid (eq_F_x), tile-width
independence, checkpoint / resume, and the host-side rejections.
Tolerances as in test_gpu_parity: FP64 relative L2 <= 1e-12 on u and C,
FP32 <= 1e-5.
"""
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


def gap_box():
    """Walled channel with two-node gaps along x and y and a block (every
    difference rule next to solid nodes)."""
    nx, ny = 26, 20
    inst = wl.channel(ny - 1, nx=nx, Wi=3.0, Sc=1e3)
    solid = np.zeros((ny, nx), np.uint8)
    solid[6:13, 8] = solid[6:13, 11] = 1
    solid[7, 14:19] = solid[10, 14:19] = 1
    solid[3:5, 21:24] = 1
    inst.solid = solid
    return inst


CASES = {
    "block_box": lambda: wl.obstacle_box(33, 20, Fx=2e-4, Fy=-5e-5, Wi=0.8),
    "disc_box_curved": lambda: wl.circle_box(37, 30, R=6.3, cx=17.2, cy=14.6, Fx=3e-4, Wi=2.0),
    "cylinder_channel_r8": lambda: wl.cylinder_channel(8, Wi=0.5, Ma=0.05),
    "gap_channel": gap_box,
}


def oracle_masked(inst, init=None):
    o = oracle_sim(inst, init=init)
    o.set_mask(inst.solid, inst.wall_q)
    return o


def run_pair(L, inst, steps, precision=0, init=None, tile_tx=0):
    sim = L.Simulation([inst], precision=precision,
                       init_fields=None if init is None else [init], tile_tx=tile_tx)
    o = oracle_masked(inst, init)
    sim.step(steps)
    o.step(steps)
    return sim, o


@pytest.mark.parametrize("case", sorted(CASES))
def test_mask_fp64_parity(lbve, case):
    """FP64 fields after 150 steps (from random initial fields) and the
    float64 totals, force on the solid included, match the oracle."""
    inst = CASES[case]()
    init = wl.random_fields(inst.nx, inst.ny, seed=31)
    sim, o = run_pair(lbve, inst, 150, init=init)
    g, r = sim.fields(0), o.fields()
    err = parity_errors(g, r)
    assert err["u"] <= FP64_TOL and err["C"] <= FP64_TOL and err["C-I"] <= 100 * FP64_TOL, err
    assert np.all(g[:, inst.solid == 1] == 0.0)
    tg, to = sim.totals(0), o.totals()
    np.testing.assert_allclose(tg[:6], to[:6], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(tg[6:12], to[6:12], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(tg[12:14], to[12:14], rtol=1e-9, atol=1e-13)
    assert np.abs(to[12:14]).max() > 0


def test_mask_fp32_parity(lbve):
    """FP32 deviation storage with a curved disc: relative L2 <= 1e-5."""
    inst = CASES["disc_box_curved"]()
    sim, o = run_pair(lbve, inst, 300, precision=1)
    err = parity_errors(sim.fields(0), o.fields())
    assert err["u"] <= FP32_TOL and err["C"] <= FP32_TOL, err


@pytest.mark.parametrize("precision", [0, 1])
def test_mask_tile_width_independent(lbve, precision):
    """Masked tiles are chosen per tile width; the fields must not change."""
    inst = CASES["disc_box_curved"]()
    ref = lbve.Simulation([inst], precision=precision)
    ref.step(70)
    for tx in (1, 5, 16, 37):
        s = lbve.Simulation([inst], precision=precision, tile_tx=tx)
        s.step(70)
        np.testing.assert_array_equal(s.fields(0), ref.fields(0), err_msg=f"tile_tx={tx}")


def test_mask_mixed_batch(lbve):
    """Masked and unmasked instances of both precisions in one handle run as
    they do alone (the per-list masked-tile and wall tables)."""
    mk = [CASES["block_box"], lambda: wl.frm(24, Wi=1.0, Re=1.0, Ma=0.05),
          CASES["cylinder_channel_r8"], lambda: wl.channel(12, nx=5, Wi=2.0),
          CASES["gap_channel"]]
    precs = [0, 1, 1, 0, 0]
    batch = lbve.Simulation([f() for f in mk], precision=precs)
    batch.step(45)
    for i, (f, p) in enumerate(zip(mk, precs)):
        alone = lbve.Simulation([f()], precision=p)
        alone.step(45)
        np.testing.assert_array_equal(batch.fields(i), alone.fields(0), err_msg=str(i))


def test_mask_save_load_resume(lbve):
    """A masked run saved and resumed continues bit-identically; a state saved
    on another mask is refused."""
    inst = CASES["cylinder_channel_r8"]()
    a = lbve.Simulation([inst], precision=0)
    a.step(37)
    state = lbve.lbve_save(a.h)
    a.step(20)
    b = lbve.Simulation([inst], precision=0)
    lbve.lbve_load(b.h, state)
    b.step(20)
    np.testing.assert_array_equal(a.fields(0), b.fields(0))
    other = wl.cylinder_channel(8, Wi=0.5, Ma=0.05, curved=False)  # same mask, other q
    c = lbve.Simulation([other], precision=0)
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_load(c.h, state)
    assert e.value.code == lbve.LBVE_ERR_GEOMETRY


def test_mask_rejections(lbve):
    """Host-side geometry checks of lbve_set_geometry / lbve_set_wall_distances
    and the adjoint's refusal of a drag loss without a mask."""
    import torch
    L = lbve
    box = CASES["block_box"]()
    # no capacity for wall nodes
    p = L.params_from(box)
    p.max_wall_nodes = 0
    n = L.lbve_workspace_bytes([p])
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    h = L.lbve_create([p], ws.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_geometry(h, 0, box.solid, n_nodes=box.n_nodes)
    assert e.value.code == L.LBVE_ERR_GEOMETRY
    L.lbve_destroy(h)
    # too small a capacity
    p.max_wall_nodes = 3
    h = L.lbve_create([p], ws.data_ptr(), L.lbve_workspace_bytes([p]),
                      torch.cuda.current_stream().cuda_stream)
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_geometry(h, 0, box.solid, n_nodes=box.n_nodes)
    assert e.value.code == L.LBVE_ERR_GEOMETRY
    L.lbve_destroy(h)
    # solid next to a flat wall; solid on both ends of a line
    ch = wl.channel(15, nx=10)
    for rows, cols in (((2,), (4,)), ((7, 7), (3, 5))):
        m = np.zeros((ch.ny, ch.nx), np.uint8)
        m[list(rows), list(cols)] = 1
        ch.solid = m
        s = None
        with pytest.raises(L.LbveError) as e:
            s = L.Simulation([ch])
        assert e.value.code == L.LBVE_ERR_GEOMETRY
        del s
    # wall distances: not a wall link, q out of range
    sim = L.Simulation([box])
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_wall_distances(sim.h, 0, [0], [1], [0.3])
    assert e.value.code == L.LBVE_ERR_GEOMETRY
    k, d, _ = box.wall_links()[0]
    with pytest.raises(L.LbveError) as e:
        L.lbve_set_wall_distances(sim.h, 0, [k], [d], [1.5])
    assert e.value.code == L.LBVE_ERR_ARG
    L.lbve_set_wall_distances(sim.h, 0, [k], [d], [0.25])
    # the adjoint covers masks and open channels (a zero loss gives a zero
    # gradient; the gradients themselves are test_gpu_adjoint_open.py's);
    # drag needs a mask
    g = torch.zeros((6, box.ny, box.nx), dtype=torch.float64, device="cuda")
    dF = torch.zeros((2, box.ny, box.nx), dtype=torch.float64, device="cuda")
    cyl = wl.cylinder_channel(4, Wi=0.5, Ma=0.05, open_x=True)
    so = L.Simulation([cyl])
    nb = L.lbve_adjoint_workspace_bytes(so.h, 0, 4)
    aws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    go = torch.zeros((6, cyl.ny, cyl.nx), dtype=torch.float64, device="cuda")
    do = torch.zeros((2, cyl.ny, cyl.nx), dtype=torch.float64, device="cuda")
    do.fill_(1.0)
    L.lbve_adjoint_step(so.h, 0, None, go.data_ptr(), 4, aws.data_ptr(), nb, do.data_ptr(),
                        cyl.n_nodes)
    assert bool((do == 0).all())
    fr = wl.frm(16, Wi=1.0, Re=1.0, Ma=0.05)
    sf = L.Simulation([fr])
    nb = L.lbve_adjoint_workspace_bytes(sf.h, 0, 4)
    aws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    gf = torch.zeros((6, 16, 16), dtype=torch.float64, device="cuda")
    df = torch.zeros((2, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(L.LbveError) as e:
        L.lbve_adjoint_step_ex(sf.h, 0, None, gf.data_ptr(), (1.0, 0.0), 4, aws.data_ptr(), nb,
                               df.data_ptr(), None, fr.n_nodes)
    assert e.value.code == L.LBVE_ERR_GEOMETRY
    del g, dF
