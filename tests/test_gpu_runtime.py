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
