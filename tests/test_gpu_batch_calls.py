"""lbve_set_geometry_many and lbve_fields_many: the batched forms of the
set-up and read-back calls give the same state as one call per instance, and
report errors per instance."""
import numpy as np
import pytest

from paper_2508_16997_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbve():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_16997_gb300 import build, lbve as L
    build.build()
    return L


def _batch():
    a = wl.frm(24, Wi=2.0, Re=1.0, Ma=0.05)
    b = wl.channel(12, nx=5, Wi=3.0)
    c = wl.obstacle_box(20, 16, Wi=0.5)
    return [a, b, c]


def _inputs(insts):
    inits = [wl.random_fields(i.nx, i.ny, seed=11 + k) for k, i in enumerate(insts)]
    forces = [wl.random_force(i.nx, i.ny, seed=5 + k, amp=2e-5) if k != 1 else None
              for k, i in enumerate(insts)]
    masks = [getattr(i, "solid", None) for i in insts]
    return masks, forces, inits


@pytest.mark.parametrize("precision", [0, 1])
def test_set_geometry_many_equals_single_calls(lbve, precision):
    """One lbve_set_geometry_many call over the batch (masks, per-node forces,
    initial fields; instances listed out of order) leaves the same state as
    one lbve_set_geometry per instance: fields bit-identical at t = 0 and
    after 40 steps."""
    insts = _batch()
    masks, forces, inits = _inputs(insts)
    n = [i.n_nodes for i in insts]
    a = lbve.Simulation(insts, precision=precision)
    b = lbve.Simulation(insts, precision=precision)
    a.step(3)
    b.step(7)
    order = [2, 0, 1]
    lbve.lbve_set_geometry_many(a.h, order, [masks[j] for j in order],
                                [forces[j] for j in order], [inits[j] for j in order],
                                n_nodes=[n[j] for j in order])
    for j in range(3):
        lbve.lbve_set_geometry(b.h, j, masks[j], forces[j], inits[j], n_nodes=n[j])
    for j in range(3):
        assert a.time(j) == b.time(j) == 0
        np.testing.assert_array_equal(a.fields(j), b.fields(j))
    a.step(40)
    b.step(40)
    for j in range(3):
        np.testing.assert_array_equal(a.fields(j), b.fields(j))
        np.testing.assert_array_equal(a.totals(j), b.totals(j))
    assert not np.any(a.status())


def test_set_geometry_many_partial_list_and_errors(lbve):
    """A list naming some instances leaves the others running; a value
    rejected on the device leaves exactly that instance uninitialised (flag
    bit 1) and the rest of the list set; a geometry rejected on the host
    stops the list there; a repeated instance changes nothing."""
    insts = _batch()
    masks, forces, inits = _inputs(insts)
    n = [i.n_nodes for i in insts]
    sim = lbve.Simulation(insts)
    sim.step(5)
    keep0 = sim.fields(0)

    # only instance 1 is reset
    lbve.lbve_set_geometry_many(sim.h, [1], None, None, [inits[1]], n_nodes=[n[1]])
    assert sim.time(0) == 5 and sim.time(1) == 0 and sim.time(2) == 5
    np.testing.assert_array_equal(sim.fields(0), keep0)

    # a repeated instance: refused before anything changes
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_set_geometry_many(sim.h, [0, 0], None, None, None, n_nodes=[n[0], n[0]])
    assert e.value.code == lbve.LBVE_ERR_ARG
    assert sim.time(0) == 5
    np.testing.assert_array_equal(sim.fields(0), keep0)

    # a NaN in the middle instance's initial fields
    bad = inits[1].copy()
    bad[2, 3, 1] = np.nan
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_set_geometry_many(sim.h, [0, 1, 2], masks, forces, [inits[0], bad, inits[2]],
                                    n_nodes=n)
    assert e.value.code == lbve.LBVE_ERR_ARG
    assert "instance 1" in str(e.value)
    flags = sim.status()
    assert flags[1] & 2 and not flags[0] & 2 and not flags[2] & 2
    assert sim.time(0) == 0 and sim.time(2) == 0
    with pytest.raises(lbve.LbveError) as e:
        sim.step(1)
    assert e.value.code == lbve.LBVE_ERR_STATE

    # a mask with no fluid at list position 1: instance 0 (position 0) is
    # set, instances 1 and 2 are not touched
    lbve.lbve_set_geometry_many(sim.h, [1], None, None, [inits[1]], n_nodes=[n[1]])
    sim.step(2)
    keep2 = sim.fields(2)
    full = np.ones((insts[2].ny, insts[2].nx), np.uint8)
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_set_geometry_many(sim.h, [0, 2, 1], [None, full, None], None, None,
                                    n_nodes=[n[0], n[2], n[1]])
    assert e.value.code == lbve.LBVE_ERR_GEOMETRY
    assert sim.time(0) == 0 and sim.time(1) == 2 and sim.time(2) == 2
    np.testing.assert_array_equal(sim.fields(2), keep2)
    sim.step(1)
    assert not np.any(sim.status())


@pytest.mark.parametrize("on_device", [False, True])
def test_fields_many_equals_single_calls(lbve, on_device):
    """lbve_fields_many writes what lbve_fields writes, to host or device
    outputs in any order; a bad instance is refused before any copy."""
    import torch
    insts = _batch()
    sim = lbve.Simulation(insts, precision=1)
    sim.step(9)
    order = [1, 2, 0]
    dev = "cuda" if on_device else "cpu"
    outs = [torch.full((6, insts[j].ny, insts[j].nx), -7.0, dtype=torch.float64, device=dev)
            for j in order]
    lbve.lbve_fields_many(sim.h, order, [t.data_ptr() for t in outs], on_device)
    torch.cuda.synchronize()
    for t, j in zip(outs, order):
        np.testing.assert_array_equal(t.cpu().numpy(), sim.fields(j))
    for t in outs:
        t.fill_(-7.0)
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_fields_many(sim.h, [0, 3], [outs[0].data_ptr(), outs[1].data_ptr()],
                              on_device)
    assert e.value.code == lbve.LBVE_ERR_ARG
    torch.cuda.synchronize()
    assert bool((outs[0] == -7.0).all())


def test_single_instance_set_geometry_in_a_large_batch(lbve):
    """lbve_set_geometry on one instance of a twelve-instance handle (its
    descriptor goes up alone) resets exactly that instance: it then evolves
    as in a handle created with the same initial fields, and its neighbours
    in the batch continue undisturbed."""
    insts = [wl.frm(12 + (j % 3), Wi=1.0 + j, Re=1.0, Ma=0.05) for j in range(12)]
    init5 = wl.random_fields(insts[5].nx, insts[5].ny, seed=55)
    a = lbve.Simulation(insts, precision=0)
    a.step(3)
    lbve.lbve_set_geometry(a.h, 5, None, insts[5].force_field, init5, n_nodes=insts[5].n_nodes)
    assert a.time(5) == 0 and a.time(4) == 3
    a.step(7)
    b = lbve.Simulation(insts, precision=0,
                        init_fields=[init5 if j == 5 else None for j in range(12)])
    b.step(7)
    np.testing.assert_array_equal(a.fields(5), b.fields(5))
    b.step(3)
    for j in (4, 6, 11):
        np.testing.assert_array_equal(a.fields(j), b.fields(j))


def test_set_geometry_many_mixed_precisions(lbve):
    """One handle holding a float64, a float32 and a float32-pair instance,
    set by one lbve_set_geometry_many (each precision's equilibrium launch
    covers its whole list), steps exactly as three one-instance handles."""
    insts = [wl.frm(20, Wi=2.0, Re=1.0, Ma=0.05), wl.channel(10, nx=7, Wi=5.0),
             wl.frm(18, Wi=1.0, Re=1.0, Ma=0.05)]
    precs = [0, 1, 2]
    inits = [wl.random_fields(i.nx, i.ny, seed=70 + k) for k, i in enumerate(insts)]
    mixed = lbve.Simulation(insts, precision=precs, init_fields=inits)
    mixed.step(25)
    for j in range(3):
        one = lbve.Simulation([insts[j]], precision=precs[j], init_fields=[inits[j]])
        one.step(25)
        np.testing.assert_array_equal(mixed.fields(j), one.fields(0))
        # the float64 tile shape may differ with the batch: totals agree to
        # the summation order's round-off
        np.testing.assert_allclose(mixed.totals(j), one.totals(0), rtol=1e-12, atol=1e-12)


def test_chunked_set_geometry_many(lbve):
    """A list of 24 instances (uploaded in chunks on the side stream) leaves
    the same state as 24 single calls, and a NaN in one instance of a later
    chunk leaves exactly that instance uninitialised."""
    insts = [wl.frm(10 + (j % 4), Wi=0.5 + j, Re=1.0, Ma=0.05) if j % 2 else
             wl.channel(6 + (j % 5), nx=3 + (j % 3), Wi=1.0 + j) for j in range(24)]
    inits = [wl.random_fields(i.nx, i.ny, seed=300 + j) for j, i in enumerate(insts)]
    n = [i.n_nodes for i in insts]
    ids = list(range(24))
    a = lbve.Simulation(insts, precision=1)
    b = lbve.Simulation(insts, precision=1)
    a.step(4)
    lbve.lbve_set_geometry_many(a.h, ids, None, [i.force_field for i in insts], inits, n_nodes=n)
    for j in ids:
        lbve.lbve_set_geometry(b.h, j, None, insts[j].force_field, inits[j], n_nodes=n[j])
    a.step(30)
    b.step(30)
    for j in ids:
        np.testing.assert_array_equal(a.fields(j), b.fields(j))
    bad = [x.copy() for x in inits]
    bad[19][5, 1, 1] = np.inf
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_set_geometry_many(a.h, ids, None, [i.force_field for i in insts], bad, n_nodes=n)
    assert e.value.code == lbve.LBVE_ERR_ARG and "instance 19" in str(e.value)
    flags = a.status()
    assert [j for j in ids if flags[j] & 2] == [19]
    assert all(a.time(j) == 0 for j in ids if j != 19)
