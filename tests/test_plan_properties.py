"""Properties of the host-side workspace planner and parameter validation,
on random parameter sets (no GPU): a valid batch gets a size that holds its
population buffers and does not depend on the tile widths; an invalid tile
width or grid is rejected with LBVE_ERR_ARG and never with a crash."""
import math

import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


@pytest.fixture(scope="module")
def L():
    from paper_2508_16997_gb300 import build, lbve
    build.build()
    return lbve


def make(L, nx, ny, periodic, precision, tile_tx=0):
    from paper_2508_16997_gb300 import workloads as wl
    Lc = nx / (2 * math.pi) if periodic else float(max(ny - 1, 1))
    inst = wl.Instance(nx, ny, periodic, 0.5, 2.0, 1.0, 1e4, 0.05, Lc)
    return L.params_from(inst, precision, tile_tx=tile_tx)


def max_width(L, precision):
    return 128 if precision == L.LBVE_FP64 else 48


instance = st.tuples(st.integers(1, 700), st.integers(3, 700), st.booleans(), st.sampled_from([0, 1]))


@settings(max_examples=60, deadline=None)
@given(batch=st.lists(instance, min_size=1, max_size=6), widths=st.data())
def test_workspace_holds_the_populations_and_ignores_tile_widths(L, batch, widths):
    base = [make(L, nx, ny, per, prec) for nx, ny, per, prec in batch]
    n0 = L.lbve_workspace_bytes(base)
    pops = sum(2 * 36 * p.nx * p.ny * (8 if p.precision == L.LBVE_FP64 else 4) for p in base)
    assert n0 >= pops
    tiled = []
    for nx, ny, per, prec in batch:
        tx = widths.draw(st.integers(1, min(max_width(L, prec), nx)))
        tiled.append(make(L, nx, ny, per, prec, tile_tx=tx))
    assert L.lbve_workspace_bytes(tiled) == n0


@settings(max_examples=40, deadline=None)
@given(inst=instance, extra=st.integers(1, 200))
def test_too_wide_tiles_are_rejected(L, inst, extra):
    nx, ny, per, prec = inst
    bad = min(max_width(L, prec), nx) + extra
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([make(L, nx, ny, per, prec, tile_tx=bad)])
    assert e.value.code == L.LBVE_ERR_ARG


@settings(max_examples=60, deadline=None)
@given(nx=st.integers(-3, 40), ny=st.integers(-3, 4), periodic=st.booleans(),
       prec=st.sampled_from([0, 1]))
def test_degenerate_grids_are_rejected(L, nx, ny, periodic, prec):
    """nx <= 0, ny <= 0 and walled grids of fewer than 3 rows are rejected;
    everything else in this range is planned."""
    p = make(L, 4, 5, periodic, prec)
    p.nx, p.ny = nx, ny
    if nx <= 0 or ny <= 0 or (not periodic and ny < 3):
        with pytest.raises(L.LbveError) as e:
            L.lbve_workspace_bytes([p])
        assert e.value.code == L.LBVE_ERR_ARG
    else:
        assert L.lbve_workspace_bytes([p]) > 0
