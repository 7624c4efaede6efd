"""The C-ABI library loads without a GPU, exports every entry point that
include/lbve.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbve.h")


@pytest.fixture(scope="module")
def L():
    from paper_2508_16997_gb300 import build, lbve
    build.build()
    return lbve


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbve_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree(L):
    assert declared_functions() == sorted(L.EXPORTED)


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbve_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    lib = L.load()
    for f in declared_functions():
        assert hasattr(lib, f)


def test_workspace_bytes_and_validation(L):
    from paper_2508_16997_gb300 import workloads as wl
    p = [L.params_from(wl.frm(64)), L.params_from(wl.channel(32), L.LBVE_FP32_DEV)]
    n = L.lbve_workspace_bytes(p)
    # two ping-pong buffers of 36 planes dominate: > 2*36*4096*8 bytes
    assert n > 2 * 36 * 4096 * 8
    bad = L.params_from(wl.frm(8))
    bad.beta = 0.0
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([bad])
    assert e.value.code == L.LBVE_ERR_ARG
    bad = L.params_from(wl.channel(8))
    bad.ny = 2
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([bad])
    assert e.value.code == L.LBVE_ERR_ARG
    bad = L.params_from(wl.frm(8))
    bad.precision = 7
    with pytest.raises(L.LbveError):
        L.lbve_workspace_bytes([bad])


def test_create_rejects_missing_workspace(L):
    from paper_2508_16997_gb300 import workloads as wl
    p = [L.params_from(wl.frm(16))]
    n = L.lbve_workspace_bytes(p)
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(p, 0, n, 0)
    assert e.value.code == L.LBVE_ERR_WORKSPACE
    with pytest.raises(L.LbveError) as e:
        L.lbve_create(p, 256, n - 1, 0)
    assert e.value.code == L.LBVE_ERR_WORKSPACE


def test_error_strings(L):
    lib = L.load()
    for code in range(0, -8, -1):
        assert lib.lbve_error_string(code)
    assert b"unknown" in lib.lbve_error_string(-99)


def test_tile_width_validation_and_layout(L):
    """tile_tx is validated on the host and never changes the workspace size."""
    from paper_2508_16997_gb300 import workloads as wl
    base = [L.params_from(wl.frm(130)), L.params_from(wl.channel(33, nx=20), L.LBVE_FP32_DEV)]
    n0 = L.lbve_workspace_bytes(base)
    for tx in (1, 3, 8, 16, 20, 48):
        p = [L.params_from(wl.frm(130), tile_tx=tx),
             L.params_from(wl.channel(33, nx=20), L.LBVE_FP32_DEV, tile_tx=min(tx, 20))]
        assert L.lbve_workspace_bytes(p) == n0
    for bad_tx in (-1, 129, 131):  # float64 tiles take up to 128
        with pytest.raises(L.LbveError) as e:
            L.lbve_workspace_bytes([L.params_from(wl.frm(256), tile_tx=bad_tx)])
        assert e.value.code == L.LBVE_ERR_ARG
    L.lbve_workspace_bytes([L.params_from(wl.frm(256), tile_tx=128)])
    with pytest.raises(L.LbveError) as e:  # float32 tiles take up to 48
        L.lbve_workspace_bytes([L.params_from(wl.frm(256), L.LBVE_FP32_DEV, tile_tx=49)])
    assert e.value.code == L.LBVE_ERR_ARG
    with pytest.raises(L.LbveError) as e:  # wider than the grid
        L.lbve_workspace_bytes([L.params_from(wl.channel(33, nx=4), tile_tx=8)])
    assert e.value.code == L.LBVE_ERR_ARG


def test_autotune_rejects_bad_arguments_on_the_host(L):
    from paper_2508_16997_gb300 import workloads as wl
    p = [L.params_from(wl.frm(64))]
    n = L.lbve_workspace_bytes(p)
    with pytest.raises(L.LbveError) as e:
        L.lbve_autotune(p, 256, n, 0, trial_steps=0)
    assert e.value.code == L.LBVE_ERR_ARG
    with pytest.raises(L.LbveError) as e:
        L.lbve_autotune(p, 0, n, 0)
    assert e.value.code == L.LBVE_ERR_WORKSPACE


def test_open_channel_validation(L):
    """open_x must be 0 or 1, and an open channel needs nx >= 5."""
    from paper_2508_16997_gb300 import workloads as wl
    p = L.params_from(wl.channel(8, nx=6))
    p.open_x = 1
    L.lbve_workspace_bytes([p])
    p.open_x = 2
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([p])
    assert e.value.code == L.LBVE_ERR_ARG
    p = L.params_from(wl.channel(8, nx=4))
    p.open_x = 1
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([p])
    assert e.value.code == L.LBVE_ERR_ARG


def test_model_validation(L):
    """model in {0, 1, 2}, L2 > 2 for the FENE models, gtilde in {0, 1}."""
    from paper_2508_16997_gb300 import workloads as wl
    for model, L2, gt, ok in ((1, 10.0, 0, True), (2, 2.5, 1, True), (3, 10.0, 0, False),
                              (1, 2.0, 0, False), (2, float("nan"), 0, False), (0, 0.0, 2, False)):
        p = L.params_from(wl.frm(16))
        p.model, p.L2, p.gtilde = model, L2, gt
        if ok:
            L.lbve_workspace_bytes([p])
        else:
            with pytest.raises(L.LbveError) as e:
                L.lbve_workspace_bytes([p])
            assert e.value.code == L.LBVE_ERR_ARG


def test_empty_degenerate_and_maximum_sizes(L):
    """An empty batch and a zero-width grid are rejected; the largest grid
    (2^25 nodes, which keeps 36 planes of indices in int32) is sized without
    overflow, and one node more is rejected."""
    from paper_2508_16997_gb300 import workloads as wl
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([])
    assert e.value.code == L.LBVE_ERR_ARG
    bad = L.params_from(wl.frm(8))
    bad.nx = 0
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([bad])
    assert e.value.code == L.LBVE_ERR_ARG
    big = L.params_from(wl.frm(8))
    big.nx, big.ny = 8192, 4096  # 2^25 nodes
    n64 = L.lbve_workspace_bytes([big])
    assert n64 > 2 * 36 * (1 << 25) * 8  # the two population buffers, float64
    big.precision = L.LBVE_FP32_DEV
    assert 2 * 36 * (1 << 25) * 4 < L.lbve_workspace_bytes([big]) < n64
    big.ny = 4097
    with pytest.raises(L.LbveError) as e:
        L.lbve_workspace_bytes([big])
    assert e.value.code == L.LBVE_ERR_ARG


def test_batched_calls_reject_bad_arguments_on_the_host(L):
    """lbve_set_geometry_many / lbve_fields_many refuse a null handle, a
    negative count or a missing list before touching the device; the binding
    refuses lists of unequal length."""
    lib = L.load()
    ids = (ctypes.c_int32 * 2)(0, 1)
    outs = (ctypes.c_void_p * 2)(None, None)
    assert lib.lbve_set_geometry_many(None, 2, ids, None, None, None) == L.LBVE_ERR_ARG
    assert lib.lbve_fields_many(None, 2, ids, outs, 0) == L.LBVE_ERR_ARG
    with pytest.raises(ValueError):
        L.lbve_set_geometry_many(None, [0, 1], [None], None, None, n_nodes=[4, 4])
    with pytest.raises(ValueError):
        L.lbve_fields_many(None, [0, 1], [0], False)
