"""lbve_field_totals_noalloc: the allocation-free variant of the totals
reduction, for callers that cannot call cudaMalloc (a framework whose
allocator owns all device memory, a latency-critical loop, a caller with a
field array but no workspace).  Its scratch is a static device array.

The test calls it through the C ABI on a field array produced by
lbve_fields(on_device=1) and compares with lbve_totals() of the same state,
on two calls in a row (the second after further steps, so the shared
scratch must not leak the first call's records).  Collected last on purpose.
"""
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


def test_noalloc_totals_match_lbve_totals(lbve):
    import torch
    inst = wl.frm(96, Wi=1.0, Re=1.0, Ma=0.1)
    init = wl.random_fields(96, 96, seed=31)
    sim = lbve.Simulation([inst], precision=lbve.LBVE_FP64, init_fields=[init])
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    for steps in (13, 29):
        sim.step(steps)
        fields = sim.fields_device(0)
        out.fill_(float("nan"))
        lbve.lbve_field_totals_noalloc(fields.data_ptr(), inst.nx, inst.ny, out.data_ptr(),
                                       stream)
        got = out.cpu().numpy()
        ref = sim.totals(0)[:6]
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("side_stream", [False, True])
def test_noalloc_totals_ragged_grid(lbve, side_stream):
    """613 x 577 = 353,701 nodes: 346 chunks, so the last chunk is partial
    and the final pass walks its strided loop (more chunks than threads).
    Run once on the current stream and once on a side stream; both calls in
    a row must agree with lbve_totals()."""
    import torch
    nx, ny = 613, 577
    inst = wl.frm(nx, Wi=1.0, Re=1.0, Ma=0.1)
    inst.ny = ny
    inst.force_field = None
    init = wl.random_fields(nx, ny, seed=47)
    sim = lbve.Simulation([inst], precision=lbve.LBVE_FP64, init_fields=[init])
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    for steps in (3, 5):
        sim.step(steps)
        fields = sim.fields_device(0)
        torch.cuda.synchronize()
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        lbve.lbve_field_totals_noalloc(fields.data_ptr(), nx, ny, out.data_ptr(),
                                       stream.cuda_stream)
        stream.synchronize()
        got = out.cpu().numpy()
        ref = sim.totals(0)[:6]
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_noalloc_rejects_oversize(lbve):
    import torch
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    dummy = torch.empty(6, dtype=torch.float64, device="cuda")
    with pytest.raises(lbve.LbveError) as e:
        lbve.lbve_field_totals_noalloc(dummy.data_ptr(), 4097, 4096, out.data_ptr(), 0)
    assert e.value.code == lbve.LBVE_ERR_ARG
    assert "static scratch limit" in str(e.value)
