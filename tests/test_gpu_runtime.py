"""Runtime features of the library on the GPU: CUDA-graph replay of step runs,
checkpoint / resume, and the reported step counts."""
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
    return [wl.frm(40, Wi=2.0, Re=1.0, Ma=0.05), wl.channel(20, nx=4, Wi=30.0),
            wl.frm(17, Wi=0.5, Re=0.1, Ma=0.01)]


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_equals_single_steps(lbve, precision):
    """lbve_step(n) with graph replays (n > 33) is bit-identical to n calls of
    lbve_step(1), including when a run starts at odd parity."""
    a = lbve.Simulation(_batch(), precision=precision)
    b = lbve.Simulation(_batch(), precision=precision)
    a.step(1)
    a.step(100)  # starts at parity 1: one direct step, then graphs
    for _ in range(101):
        b.step(1)
    for i in range(3):
        np.testing.assert_array_equal(a.fields(i), b.fields(i))
        np.testing.assert_array_equal(a.totals(i)[:6], b.totals(i)[:6])
    assert a.time(0) == b.time(0) == 101


@pytest.mark.parametrize("precision", [0, 1])
def test_save_load_bit_exact_resume(lbve, precision):
    """A run saved at step 37 and resumed in a fresh handle continues
    bit-identically; a state from a different handle shape is rejected."""
    insts = _batch()
    inits = [wl.random_fields(i.nx, i.ny, seed=7 + k) for k, i in enumerate(insts)]
    a = lbve.Simulation(insts, precision=precision, init_fields=inits)
    a.step(37)
    state = lbve.lbve_save(a.h)
    a.step(50)
    b = lbve.Simulation(_batch(), precision=precision)  # different initial state
    lbve.lbve_load(b.h, state)
    assert b.time(0) == 37
    b.step(50)
    for i in range(3):
        np.testing.assert_array_equal(a.fields(i), b.fields(i))
    c = lbve.Simulation(_batch()[:2], precision=precision)
    with pytest.raises(lbve.LbveError):
        lbve.lbve_load(c.h, state)


def _ragged_batch():
    # ragged in x and y for every tile width; walled and periodic; a force field
    f = wl.frm(70, Wi=2.0, Re=1.0, Ma=0.05)
    return [f, wl.channel(37, nx=45, Wi=30.0), wl.frm(17, Wi=0.5, Re=0.1, Ma=0.01)]


@pytest.mark.parametrize("precision", [0, 1])
def test_tile_width_does_not_change_fields(lbve, precision):
    """Each node's update is independent of the tiling: the fields after 60
    steps are bit-identical for every tile width, and the float64 totals
    (whose summation follows the tiles) agree to rounding."""
    insts = _ragged_batch()
    inits = [wl.random_fields(i.nx, i.ny, seed=11 + k) for k, i in enumerate(insts)]
    ref = lbve.Simulation(insts, precision=precision, init_fields=inits)
    ref.step(60)
    for tx in (1, 5, 8, 16, 48):
        widths = [min(tx, i.nx) for i in insts]
        s = lbve.Simulation(insts, precision=precision, init_fields=inits, tile_tx=widths)
        s.step(60)
        for i in range(len(insts)):
            np.testing.assert_array_equal(s.fields(i), ref.fields(i), err_msg=f"tile_tx={tx}")
            t0, t1 = ref.totals(i), s.totals(i)
            np.testing.assert_allclose(t1[:6], t0[:6], rtol=1e-13, atol=1e-13 * np.abs(t0[:6]).max())


def test_autotune_picks_admissible_widths(lbve):
    """lbve_autotune returns one admissible width per instance, the same for
    instances of one class, and the tuned batch reproduces the default one."""
    insts = [wl.frm(128), wl.frm(128, Wi=2.0), wl.channel(64, nx=4), wl.frm(96)]
    s = lbve.Simulation(insts, precision=1, autotune=16)
    for tx, inst in zip(s.tile_tx, insts):
        assert 1 <= tx <= min(128, inst.nx)
    assert s.tile_tx[0] == s.tile_tx[1]
    assert s.tile_tx[2] == 4
    ref = lbve.Simulation(insts, precision=1)
    s.step(40)
    ref.step(40)
    for i in range(len(insts)):
        np.testing.assert_array_equal(s.fields(i), ref.fields(i))


def test_fp64_cta_sizes_bit_identical(lbve):
    """The float64 CTA size follows the batch (one-warp tiles for a 64^2 mill
    or the five Wi-sweep channels, 64 and 256 threads when a wider tile is
    asked for): the fields are bit-identical whichever runs them."""
    for insts in ([wl.frm(64, Wi=2.0, Re=1.0, Ma=0.05)],
                  [wl.channel(64, nx=4, Wi=w) for w in (1.0, 10.0, 100.0, 1e3, 1e4)]):
        inits = [wl.random_fields(i.nx, i.ny, seed=5 + k, du=1e-3, dA=0.05)
                 for k, i in enumerate(insts)]
        runs = []
        for tx in (0, 32, 64):
            widths = [min(tx, i.nx) for i in insts]
            s = lbve.Simulation(insts, precision=lbve.LBVE_FP64, init_fields=inits, tile_tx=widths)
            s.step(50)
            runs.append([s.fields(i) for i in range(len(insts))])
        for r in runs[1:]:
            for a, b in zip(r, runs[0]):
                np.testing.assert_array_equal(a, b)


def test_profile_times_every_launch(lbve):
    """lbve_profile arms per-launch events for the plain step kernel: every
    launch of the next step calls is timed up to the cap, while armed the
    steps run as direct launches with fields bit-identical to a graph-replayed
    run, and disarming releases the events."""
    insts = _batch()
    a = lbve.Simulation(insts, precision=1)
    b = lbve.Simulation(insts, precision=1)
    lbve.lbve_profile(a.h, 50)
    a.step(7)
    n, tot, lo, hi = lbve.lbve_profile_read(a.h, lbve.LBVE_FP32_DEV)
    assert n == 6 and tot > 0 and 0 < lo <= hi <= tot  # 6 ordinary steps
    n, tot, lo, hi = lbve.lbve_profile_read(a.h, lbve.LBVE_FP32_DEV, final_step=True)
    assert n == 1 and tot > 0 and lo == hi == tot
    assert lbve.lbve_profile_read(a.h, lbve.LBVE_FP64)[0] == 0  # no float64 instance
    a.step(70)  # 44 more timed ordinary launches, the rest untimed
    assert lbve.lbve_profile_read(a.h, lbve.LBVE_FP32_DEV)[0] == 50
    assert lbve.lbve_profile_read(a.h, lbve.LBVE_FP32_DEV, final_step=True)[0] == 2
    b.step(77)  # two graph replays of 32 steps
    for i in range(len(insts)):
        np.testing.assert_array_equal(a.fields(i), b.fields(i))
    lbve.lbve_profile(a.h, 0)
    assert lbve.lbve_profile_read(a.h, lbve.LBVE_FP32_DEV)[0] == 0
    with pytest.raises(lbve.LbveError):
        lbve.lbve_profile(a.h, -1)
