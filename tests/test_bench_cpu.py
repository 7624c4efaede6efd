"""Host logic of bench.py, on the CPU: the batched-mix recipe, the
algorithmic bytes per lattice update, whole-job MLUPS, the per-rank seeds
and the rule that a profile summary taken on other kernel sources reads as
missing (null) rather than as a stale number."""
import os

import numpy as np
import pytest

import bench


def test_batched_mix_recipe():
    """256 instances: 128 channels (nx = 4, H ~ U{32..512}, walls on rows 0
    and H) then 128 periodic four-roll mills (N ~ U{64..512}); Wi in
    [1, 1e4], beta in [0.1, 0.9]; about 12.7 M nodes; the same seeds give the
    same mix."""
    insts = bench.workload(0, 256)
    assert len(insts) == 256
    ch, frm = insts[:128], insts[128:]
    assert all(i.kind == "channel" and i.nx == 4 and not i.periodic_y for i in ch)
    assert all(32 <= i.ny - 1 <= 512 for i in ch)
    assert all(i.kind == "frm" and i.nx == i.ny and i.periodic_y for i in frm)
    assert all(64 <= i.nx <= 512 for i in frm)
    assert all(1.0 <= i.Wi <= 1e4 and 0.1 <= i.beta <= 0.9 for i in insts)
    nodes = sum(i.n_nodes for i in insts)
    assert 12.0e6 < nodes < 13.5e6
    again = bench.workload(0, 256)
    assert [(i.nx, i.ny, i.Wi, i.beta) for i in again] == [(i.nx, i.ny, i.Wi, i.beta) for i in insts]


def test_ranks_draw_independent_mixes():
    """Weak scaling: each rank runs its own seeded mix of the same recipe."""
    a, b = bench.workload(0, 16), bench.workload(1, 16)
    assert bench.rank_seed(0) != bench.rank_seed(1)
    assert [(i.nx, i.ny, i.Wi) for i in a] != [(i.nx, i.ny, i.Wi) for i in b]


def test_bytes_per_lattice_update_and_job_value():
    """82 scalars per update (36 populations and 5 history values, each read
    and written once): 328 B in FP32, 656 B in FP64; 8 / 16 B more with a
    per-node force field.  MLUPS = all ranks' updates over the slowest time."""
    from paper_2508_16997_gb300 import workloads as wl
    ch, mill = wl.channel(32), wl.frm(64)
    assert mill.force_field is not None and ch.force_field is None
    assert bench.bytes_per_lu(ch, 4) == 328 and bench.bytes_per_lu(ch, 8) == 656
    assert bench.bytes_per_lu(mill, 4) == 336 and bench.bytes_per_lu(mill, 8) == 672
    assert bench.job_value(2_000_000, 1000, 0.5) == pytest.approx(4000.0)


def test_profile_values_follow_the_kernel_sources(monkeypatch, tmp_path):
    """A committed summary counts only while its recorded source hash is the
    hash of the current step-kernel sources; otherwise every derived key is
    None."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "roofline_traffic.txt").write_text(
        "# comment\nsources_sha256 abc\ndram_bytes_per_launch 123\n")
    (tmp_path / "profiles" / "step_kernel_flop_count.txt").write_text(
        "sources_sha256 abc\nflop_per_lu 600\nfp32_peak_tflops 80\n"
        "fp64_inst_per_lu 400\nfp64_peak_ginst 600\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: "abc")
    assert bench.measured_traffic() == 123.0
    f = bench.measured_flops(1000.0)
    assert f["achieved"] == pytest.approx(0.6) and f["frac"] == pytest.approx(0.6 / 80)
    p = bench.measured_fp64_pipe(1000.0)
    assert p["achieved"] == pytest.approx(400.0) and p["bound"] == "alu"
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: "changed")
    assert bench.measured_traffic() is None
    assert bench.measured_flops(1000.0) is None
    assert bench.measured_fp64_pipe(1000.0) is None


def test_committed_profiles_parse():
    """The committed summaries carry every key the bench reads."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    keys = {}
    for name in ("roofline_traffic.txt", "step_kernel_flop_count.txt"):
        with open(os.path.join(root, "profiles", name)) as f:
            for line in f:
                if line.strip() and not line.startswith("#"):
                    k, v = line.split(None, 1)
                    keys[k] = v.strip()
    for k in ("dram_bytes_per_launch", "flop_per_lu", "fp32_peak_tflops", "fp64_inst_per_lu",
              "fp64_peak_ginst"):
        assert np.isfinite(float(keys[k])) and float(keys[k]) > 0, k
    assert len(keys["sources_sha256"]) == 64
