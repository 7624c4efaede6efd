#!/usr/bin/env python
"""Benchmark of the coupled viscoelastic LBM step on GB300.

Workload: the batched mix of force-driven Oldroyd-B Poiseuille channels and
simplified four-roll mills (256 seeded instances of uneven sizes, Wi and
beta), all advanced together by one launch per time step, FP32-deviation
storage with float64 reductions.  One bench "step" is one coupled time step
of every instance.  The metric is MLUPS (one lattice update = all four
lattices at one node), whole job.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled-LBM MLUPS & % HBM roofline; FP32/batched vs plain FP64 at stated error"
UNIT = "MLUPS"
BASE_SEED = 20250823
N_INSTANCES = 256
SCALARS_PER_LU = 82  # 36 populations + 5 history values, read and written
ADJOINT_SEED = 5


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--instances", type=int, default=N_INSTANCES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--cylinder-steps", type=int, default=2000)
    ap.add_argument("--frm64-steps", type=int, default=2000)
    ap.add_argument("--frm-large-steps", type=int, default=20,
                    help="timed steps of the four-roll mill at 2048^2 and 4096^2 (0: skip)")
    ap.add_argument("--error-steps", type=int, default=2000)
    return ap.parse_args()


def rank_seed(rank: int) -> int:
    """Base seed of a rank's batch: every rank runs its own independent mix
    (weak scaling, no data exchange between ranks)."""
    return BASE_SEED + 100003 * rank


def workload(rank: int, n: int):
    from paper_2508_16997_gb300 import workloads as wl
    return wl.batch_mix(n=n, base_seed=rank_seed(rank))


def workspace_bytes(insts, precision: int = 1) -> int:
    """Device workspace a rank's batch needs (lbve_workspace_bytes, a host-only
    call of the library): the plan of its buffers in HBM."""
    from paper_2508_16997_gb300 import lbve
    return lbve.lbve_workspace_bytes([lbve.params_from(i, precision) for i in insts])


def job_value(job_nodes: int, steps: int, seconds_max: float) -> float:
    """Whole-job MLUPS: the lattice updates of all ranks (job_nodes nodes in
    total, each advanced `steps` steps) over the slowest rank's time."""
    return job_nodes * steps / seconds_max / 1e6


def bytes_per_lu(inst, elem: int) -> int:
    """Algorithmic HBM bytes of one lattice update: 82 scalars (36 populations
    and 5 history values, each read once and written once) plus the 2 force
    components when the instance has a per-node force field."""
    return elem * (SCALARS_PER_LU + (2 if inst.force_field is not None else 0))


def workload_desc(insts, total_nodes):
    n_ch = sum(1 for i in insts if i.kind == "channel")
    return {
        "workload": (f"batched mix: {n_ch} Oldroyd-B Poiseuille channels (nx=4, H~U{{32..512}}) + "
                     f"{len(insts) - n_ch} four-roll mills (N~U{{64..512}}), Wi=10^U(0,4), "
                     f"beta~U(0.1,0.9), seeds {BASE_SEED}+i"),
        "instances": len(insts),
        "nodes_per_gpu": total_nodes,
        "storage": "fp32 deviations, fp64 totals",
        "l2": "inputs larger than L2 (working set >> 129 MB), no flush needed",
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines: list[str] = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def wait_first(self, timeout: float = 3.0):
        """Wait until the first sample has arrived (or the sampler is absent)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.02)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("lbve_step.cuh", "lbve_df32.cuh", "lbve_kernels.cu", "lbve_internal.h"):
        with open(os.path.join(ROOT, "paper_2508_16997_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profile_values(name):
    """Key/value lines of a committed profile summary, or None when the
    kernel sources changed since the capture it records."""
    try:
        vals = {}
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if line.startswith("#") or not line.strip():
                    continue
                k, v = line.split(None, 1)
                vals[k] = v.strip()
    except (OSError, ValueError):
        return None
    if vals.get("sources_sha256") != kernel_sources_sha256():
        return None
    return vals


def measured_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    capture, or None when the kernel sources changed since the capture."""
    vals = profile_values("roofline_traffic.txt")
    try:
        return float(vals["dram_bytes_per_launch"])
    except (TypeError, KeyError, ValueError):
        return None


def measured_flops(mlups):
    """Floating-point work of the float32 step kernel: flops per lattice
    update counted by ncu (fadd + fmul + 2 ffma per node), the throughput
    they make at `mlups`, and the fraction of the FP32 (non-tensor) peak
    derived from 152 SMs x 128 lanes x 2 flops x 2.07 GHz.  None when the
    kernel changed since the count."""
    vals = profile_values("step_kernel_flop_count.txt")
    try:
        per_lu, peak = float(vals["flop_per_lu"]), float(vals["fp32_peak_tflops"])
    except (TypeError, KeyError, ValueError):
        return None
    achieved = per_lu * mlups * 1e6 / 1e12
    return {"per_lu": per_lu, "achieved": achieved, "unit": "TFLOP/s", "peak": peak,
            "peak_kind": "derived from unit counts and the maximum SM clock",
            "frac": achieved / peak,
            "source": "ncu thread-instruction counters of step_kernel<float> on four-roll "
                      "mills 512^2 x 8"}


def measured_fp64_pipe(mlups):
    """The float64 step kernel against its FP64 pipe: FP64 instructions per
    lattice update counted by ncu (dadd + dmul + dfma per node), the
    instruction rate they make at `mlups`, and the fraction of the pipe's
    peak derived from 152 SMs x 2 FP64 instructions per clock x 2.07 GHz.
    None when the kernel changed since the count."""
    vals = profile_values("step_kernel_flop_count.txt")
    try:
        per_lu = float(vals["fp64_inst_per_lu"])
        peak = float(vals["fp64_peak_ginst"])
    except (TypeError, KeyError, ValueError):
        return None
    achieved = per_lu * mlups * 1e6 / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G FP64 inst/s",
            "frac": achieved / peak, "inst_per_lu": per_lu,
            "peak_kind": "derived from unit counts and the maximum SM clock",
            "source": "ncu thread-instruction counters of step_kernel<double> on four-roll "
                      "mills 512^2 x 8"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(v: float, world: int, device: str = "cpu") -> float:
    """Maximum of v over the ranks of the default process group (v itself
    when running alone)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(v: float, world: int, device: str = "cpu") -> float:
    """Sum of v over the ranks of the default process group."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_sample(insts, budget_nodes: int):
    """Smallest instances of the mix, in order, up to budget_nodes nodes."""
    chosen, total = [], 0
    for inst in sorted(insts, key=lambda i: i.n_nodes):
        if chosen and total + inst.n_nodes > budget_nodes:
            break
        chosen.append(inst)
        total += inst.n_nodes
    return chosen, total


def time_oracle(sample, steps: int):
    """Oracle wall time for `steps` steps of every sample instance."""
    from oracle import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_helpers import oracle_sim
    oracle.build()
    sims = [oracle_sim(inst) for inst in sample]
    t0 = time.perf_counter()
    for s in sims:
        s.step(steps)
    return time.perf_counter() - t0


def _oracle_worker(job):
    """Pool worker: step a share of the sample's instances on the oracle and
    return the seconds spent stepping (set-up excluded)."""
    insts, steps = job
    from oracle import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_helpers import oracle_sim
    oracle.build()
    sims = [oracle_sim(inst) for inst in insts]
    t0 = time.perf_counter()
    for s in sims:
        s.step(steps)
    return time.perf_counter() - t0


def time_oracle_all_cores(sample, steps: int):
    """The same oracle runs spread over every host core: the independent
    instances are dealt round-robin (largest first) to one process per core,
    started with spawn (this process already holds a CUDA context).  Returns
    (seconds of the slowest worker, workers)."""
    import multiprocessing as mp
    workers = max(1, min(os.cpu_count() or 1, len(sample)))
    shares = [[] for _ in range(workers)]
    for j, inst in enumerate(sorted(sample, key=lambda i: -i.n_nodes)):
        shares[j % workers].append(inst)
    with mp.get_context("spawn").Pool(workers) as pool:
        secs = pool.map(_oracle_worker, [(sh, steps) for sh in shares])
    return max(secs), workers


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    insts = workload(0, args.instances)
    total_steps = args.warmup + args.steps
    # size each step so that the whole run is about a minute of oracle work
    budget = max(1, int(60.0 * 1.0e6 / total_steps))
    sample, nodes = cpu_sample(insts, budget)
    from oracle import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle_helpers import oracle_sim
    oracle.build()
    sims = [oracle_sim(inst) for inst in sample]
    for s in sims:
        s.step(args.warmup)
    t0 = time.perf_counter()
    for s in sims:
        s.step(args.steps)
    dt = time.perf_counter() - t0
    value = nodes * args.steps / dt / 1e6
    desc = f"oracle FP64, {len(sample)} smallest instances of the mix ({nodes} nodes) per step"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": workload_desc(insts, sum(i.n_nodes for i in insts)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_16997_gb300 import build as b, lbve
    if rank == 0 or world == 1:
        b.build()
    if world > 1:
        torch.distributed.barrier()
    b.build()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, world, device="cuda")

    insts = workload(rank, args.instances)
    total_nodes = sum(i.n_nodes for i in insts)
    job_nodes = int(reduce_sum(float(total_nodes), world, device="cuda"))
    stream = torch.cuda.current_stream()
    K, W = args.steps, args.warmup

    # ---- headline: FP32-deviation batch, inputs resident in HBM -------------
    # The clock sampler starts before the warm-up, so that its start-up does
    # not leave the GPU idle right before the timed steps.  The library times
    # every launch of the step kernel in the timed region with CUDA events on
    # the stream it launches on (lbve_profile), next to the whole region.
    sim = lbve.Simulation(insts, precision=lbve.LBVE_FP32_DEV)
    ws_bytes = sim.nbytes
    with ClockSampler(local) as clk:
        clk.wait_first()
        sim.step(W)
        torch.cuda.synchronize()
        barrier()
        lbve.lbve_profile(sim.h, K)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    # the dominant kernel: the ordinary (non-final) step; the last step of the
    # call is a kernel of its own that also writes the float64 fields
    n_timed, k_tot, k_min, k_max = lbve.lbve_profile_read(sim.h, lbve.LBVE_FP32_DEV)
    n_fin, f_tot, _, _ = lbve.lbve_profile_read(sim.h, lbve.LBVE_FP32_DEV, final_step=True)
    lbve.lbve_profile(sim.h, 0)
    kernel_ms = max_over_ranks(k_tot / max(n_timed, 1))
    final_ms = max_over_ranks(f_tot / max(n_fin, 1))
    flags = sim.status()
    value = job_value(job_nodes, K, ms / 1e3)
    bytes_launch = sum(i.n_nodes * bytes_per_lu(i, 4) for i in insts)
    achieved = bytes_launch / (kernel_ms / 1e3) / 1e9
    achieved_step = bytes_launch / (ms / 1e3 / K) / 1e9
    peak, peak_kind = measured_peaks()

    # ---- end to end through the C ABI with host buffers --------------------
    # lbve_set_geometry_many uploads every instance's state (pinned host
    # force field and initial fields) and initialises it, lbve_step(K)
    # advances the batch, lbve_fields_many copies every instance's fields
    # back to pinned host memory.  The upload happens once per K steps: bytes
    # are stated per call and per step (per call / K).
    pinned_force = [None if i.force_field is None else
                    torch.from_numpy(np.ascontiguousarray(i.force_field)).pin_memory()
                    for i in insts]
    pinned_init = []
    for i in insts:
        f = np.zeros((6, i.ny, i.nx))
        f[0] = 1.0
        f[3] = 1.0
        f[5] = 1.0
        pinned_init.append(torch.from_numpy(f).pin_memory())
    pinned_out = [torch.empty((6, i.ny, i.nx), dtype=torch.float64).pin_memory() for i in insts]
    h2d = sum(t.numel() * 8 for t in pinned_init) + sum(
        t.numel() * 8 for t in pinned_force if t is not None)
    d2h = sum(t.numel() * 8 for t in pinned_out)
    ids = list(range(len(insts)))
    force_np = [None if t is None else t.numpy() for t in pinned_force]
    init_np = [t.numpy() for t in pinned_init]
    out_ptrs = [t.data_ptr() for t in pinned_out]
    n_nodes = [i.n_nodes for i in insts]

    def e2e_pass():
        t0 = time.perf_counter()
        lbve.lbve_set_geometry_many(sim.h, ids, None, force_np, init_np, n_nodes=n_nodes)
        t1 = time.perf_counter()
        sim.step(K)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        lbve.lbve_fields_many(sim.h, ids, out_ptrs, False)
        torch.cuda.synchronize()
        return t0, t1, t2, time.perf_counter()

    e2e_pass()  # warm-up: the first touches of the pinned buffers are not timed
    torch.cuda.synchronize()
    barrier()
    t0, t1, t2, t3 = e2e_pass()
    e2e_s = max_over_ranks(t3 - t0)
    e2e_value = job_value(job_nodes, K, e2e_s)
    e2e_parts = {"upload_and_init": t1 - t0, "steps": t2 - t1, "download": t3 - t2}

    # ---- plain FP64 on the same mix, and the FP32 error against it ---------
    # FP64 is timed over K64 steps (per-launch kernel time alongside); both
    # precisions then run to E steps from the same initial state and the
    # FP32 fields are compared with the FP64 ones, per decade of Wi.
    K64 = max(1, min(K, 200))
    E = max(args.error_steps, W + K64)
    sim64 = lbve.Simulation(insts, precision=lbve.LBVE_FP64)
    sim64.step(W)
    torch.cuda.synchronize()
    barrier()
    lbve.lbve_profile(sim64.h, K64)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    sim64.step(K64)
    f1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(f0.elapsed_time(f1))
    n64, k64_tot, _, _ = lbve.lbve_profile_read(sim64.h, lbve.LBVE_FP64)
    lbve.lbve_profile(sim64.h, 0)
    kernel_ms64 = max_over_ranks(k64_tot / max(n64, 1))
    value64 = job_value(job_nodes, K64, ms64 / 1e3)
    sim64.step(E - W - K64)
    for j in range(len(insts)):  # FP32 run from the same initial state, same step count
        lbve.lbve_set_geometry(sim.h, j, None, insts[j].force_field, None,
                               n_nodes=insts[j].n_nodes)
    sim.step(E)
    flags64 = sim64.status()
    bins = {"1-10": (1.0, 10.0), "10-100": (10.0, 100.0), "100-1e3": (100.0, 1e3),
            "1e3-1e4": (1e3, 1e4 + 1)}
    per_bin = {k: {"u": 0.0, "C": 0.0, "instances": 0, "within_1e-5": 0} for k in bins}
    per_kind = {k: {"u": 0.0, "C": 0.0, "instances": 0, "within_1e-5": 0}
                for k in ("channel", "frm")}
    err_all, err_le100 = 0.0, 0.0
    for j, inst in enumerate(insts):
        if flags64[j]:
            continue
        a = sim.fields_device(j)
        r = sim64.fields_device(j)
        eu = float(torch.linalg.vector_norm(a[1:3] - r[1:3]) / torch.linalg.vector_norm(r[1:3]))
        eC = float(torch.linalg.vector_norm(a[3:6] - r[3:6]) / torch.linalg.vector_norm(r[3:6]))
        e = max(eu, eC)
        err_all = max(err_all, e)
        if inst.Wi <= 100:
            err_le100 = max(err_le100, e)
        for k, (lo, hi) in bins.items():
            if lo <= inst.Wi < hi:
                b_ = per_bin[k]
                b_["u"] = max(b_["u"], eu)
                b_["C"] = max(b_["C"], eC)
                b_["instances"] += 1
                b_["within_1e-5"] += int(e <= 1e-5)
        if inst.kind in per_kind:
            b_ = per_kind[inst.kind]
            b_["u"] = max(b_["u"], eu)
            b_["C"] = max(b_["C"], eC)
            b_["instances"] += 1
            b_["within_1e-5"] += int(e <= 1e-5)
    err_all = max_over_ranks(err_all)
    err_le100 = max_over_ranks(err_le100)

    # ---- float32 pairs (LBVE_DF32) on the same mix ---------------------------
    # timed over K64 steps like FP64, then run to E steps from the same initial
    # state and compared with the FP64 fields of step E
    simd = lbve.Simulation(insts, precision=lbve.LBVE_DF32)
    simd.step(W)
    torch.cuda.synchronize()
    barrier()
    lbve.lbve_profile(simd.h, K64)
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    simd.step(K64)
    d1.record(stream)
    torch.cuda.synchronize()
    msd = max_over_ranks(d0.elapsed_time(d1))
    nd, kd_tot, _, _ = lbve.lbve_profile_read(simd.h, lbve.LBVE_DF32)
    lbve.lbve_profile(simd.h, 0)
    kernel_msd = max_over_ranks(kd_tot / max(nd, 1))
    valued = job_value(job_nodes, K64, msd / 1e3)
    simd.step(E - W - K64)
    errd = {"channel": 0.0, "frm": 0.0}
    for j, inst in enumerate(insts):
        if flags64[j]:
            continue
        a = simd.fields_device(j)
        r = sim64.fields_device(j)
        eu = float(torch.linalg.vector_norm(a[1:3] - r[1:3]) / torch.linalg.vector_norm(r[1:3]))
        eC = float(torch.linalg.vector_norm(a[3:6] - r[3:6]) / torch.linalg.vector_norm(r[3:6]))
        if inst.kind in errd:
            errd[inst.kind] = max(errd[inst.kind], eu, eC)
    errd = {k: max_over_ranks(v) for k, v in errd.items()}
    bytes_df = sum(i.n_nodes * bytes_per_lu(i, 8) for i in insts)
    del simd

    # ---- adjoint: the 512^2 four-roll mill, FP32, sqrt(T) checkpointing ----
    # loss L = 1/2 sum |u(T) - u_target|^2, the target from a run with the
    # seeded perturbed force F + 0.01 F0 xi, xi ~ N(0, 1) per node and component
    adj = None
    if args.adjoint_steps > 0:
        import copy
        from paper_2508_16997_gb300 import workloads as wl
        Ta = args.adjoint_steps
        fi = wl.frm(512, Wi=5.0)
        F0 = float(np.abs(fi.force_field).max())
        xi = np.random.default_rng(ADJOINT_SEED).standard_normal(fi.force_field.shape)
        ft = copy.copy(fi)
        ft.force_field = fi.force_field + 0.01 * F0 * xi
        tsim = lbve.Simulation([ft], precision=lbve.LBVE_FP32_DEV)
        tsim.step(Ta)
        target = tsim.fields_device(0).clone()
        del tsim
        asim = lbve.Simulation([fi], precision=lbve.LBVE_FP32_DEV)
        asim.step(Ta)
        fields = asim.fields_device(0)
        g = torch.zeros_like(fields)
        g[1:3] = fields[1:3] - target[1:3]  # dL/du
        loss = 0.5 * float((g[1:3] ** 2).sum())
        nbytes = lbve.lbve_adjoint_workspace_bytes(asim.h, 0, Ta)
        aws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        dF = torch.empty((2, 512, 512), dtype=torch.float64, device="cuda")
        lbve.lbve_adjoint_step(asim.h, 0, None, g.data_ptr(), Ta, aws.data_ptr(), nbytes,
                               dF.data_ptr(), fi.n_nodes)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbve.lbve_adjoint_step(asim.h, 0, None, g.data_ptr(), Ta, aws.data_ptr(), nbytes,
                               dF.data_ptr(), fi.n_nodes)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        # the same gradient with every forward state stored (no recomputation),
        # when the device has room for it
        store_all = None
        nb1 = lbve.lbve_adjoint_workspace_bytes_interval(asim.h, 0, Ta, 1)
        del aws
        if torch.cuda.mem_get_info()[0] > 1.1 * nb1:
            aws1 = torch.empty(nb1, dtype=torch.uint8, device="cuda")
            dF1 = torch.empty_like(dF)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            lbve.lbve_adjoint_step(asim.h, 0, None, g.data_ptr(), Ta, aws1.data_ptr(), nb1,
                                   dF1.data_ptr(), fi.n_nodes)
            torch.cuda.synchronize()
            dt1 = time.perf_counter() - t1
            store_all = {"seconds": dt1, "ms_per_reversed_step": 1e3 * dt1 / Ta,
                         "workspace_bytes": nb1,
                         "gradient_identical": bool(torch.equal(dF1, dF))}
            del aws1, dF1
        adj = {"workload": "four-roll mill 512^2, beta 0.5, Wi 5, FP32; loss 1/2 |u(T) - u_target|^2, "
                           f"target from the force F + 0.01 F0 xi (xi ~ N(0,1), seed {ADJOINT_SEED})",
               "steps": Ta, "checkpoint_interval": int(np.ceil(np.sqrt(Ta))),
               "seconds": dt, "ms_per_reversed_step": 1e3 * dt / Ta,
               "loss": loss, "grad_norm": float(torch.linalg.vector_norm(dF)),
               "workspace_bytes": nbytes,
               "includes": "forward recompute from the initial fields (checkpoints + segments) "
                           "and the reverse sweep",
               "store_all_states": store_all}
        del asim

    # ---- cylinder in a channel (solid mask, curved walls, drag) -----------
    cyl = None
    if args.cylinder_steps > 0:
        cyl = bench_cylinder(args.cylinder_steps, stream)

    # ---- the small four-roll mill as specified (64^2, FP64, from rest) ------
    c1, c1_fields = None, None
    if args.frm64_steps > 0:
        c1, c1_fields = bench_frm64(args.frm64_steps, stream)

    # ---- the same four-roll mill on large grids: roofline of one instance --
    frm_large = None
    if args.frm_large_steps > 0:
        frm_large = bench_frm_large(args.frm_large_steps, stream)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_desc(insts, total_nodes), workspace_bytes_per_gpu=ws_bytes),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": measured_traffic(),
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "kernel": "step_kernel<float, step, non-final> (one launch per step; "
                               "K - 1 of the K launches)",
                     "kernel_ms": kernel_ms, "kernel_ms_min": k_min, "kernel_ms_max": k_max,
                     "launches_timed": n_timed,
                     "final_step_kernel_ms": final_ms,
                     "timing": "CUDA events around every step-kernel launch of the timed "
                               "region, on the stream it is launched on (lbve_profile)",
                     "whole_step": {"ms": ms / K, "achieved": achieved_step,
                                    "frac": achieved_step / peak,
                                    "includes": "the last step's float64 field write and the "
                                                "end-of-call reduction"}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
                "d2h_bytes_per_step": d2h / K, "h2d_bytes_per_call": h2d,
                "d2h_bytes_per_call": d2h, "steps_per_call": K,
                "seconds": e2e_parts,
                "region": "once per K steps: lbve_set_geometry_many (pinned host force + "
                          "initial fields of every instance, one synchronisation), "
                          "lbve_step(K), lbve_fields_many (every instance to pinned host, "
                          "one synchronisation)"},
        "flops": measured_flops(value),
        "gpu_launches": K + 1,
        "clocks": clocks,
        "fp64_plain": {"value": value64, "unit": UNIT, "steps": K64, "ms_per_step": ms64 / K64,
                       "kernel_ms": kernel_ms64,
                       "speedup_fp32_over_fp64": value / value64,
                       "roofline": measured_fp64_pipe(value64)},
        "df32": {"value": valued, "unit": UNIT, "steps": K64, "ms_per_step": msd / K64,
                 "kernel_ms": kernel_msd, "speedup_over_fp64": valued / value64,
                 "roofline": {"bound": "hbm", "achieved": bytes_df / (kernel_msd / 1e3) / 1e9,
                              "peak": peak, "unit": "GB/s",
                              "frac": bytes_df / (kernel_msd / 1e3) / 1e9 / peak,
                              "algorithmic_bytes_per_launch": bytes_df},
                 "vs_fp64_rel_l2": {"steps": E, "max_per_kind": errd},
                 "storage": "float32 pairs (hi + lo), 8 B per value; float32-pipe arithmetic"},
        "fp32_vs_fp64_rel_l2": {"max_all": err_all, "max_Wi_le_100": err_le100,
                                "per_Wi": per_bin, "per_kind": per_kind, "steps": E,
                                "target_Wi_le_100": 1e-5},
        "nonfinite_instances": int((flags != 0).sum()),
    }
    if adj is not None:
        line["adjoint"] = adj
    if cyl is not None:
        line["cylinder"] = cyl
    if c1 is not None:
        line["frm64"] = c1
    if frm_large is not None:
        line["frm_large"] = frm_large
    if world == 1 and not args.no_cpu_baseline:
        sample, nodes = cpu_sample(insts, 50000)
        steps_cpu = 200
        dt = time_oracle(sample, steps_cpu)
        line["cpu_baseline"] = {
            "value": nodes * steps_cpu / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 oracle, {len(sample)} smallest instances of the mix "
                      f"({nodes} nodes) x {steps_cpu} steps, single thread"}
        # the same sample on every host core (independent instances, one
        # process per core): a larger sample so that each core has work
        sample_all, nodes_all = cpu_sample(insts, 50000 * (os.cpu_count() or 1))
        dt_all, workers = time_oracle_all_cores(sample_all, steps_cpu)
        line["cpu_baseline_all_cores"] = {
            "value": nodes_all * steps_cpu / dt_all / 1e6, "unit": UNIT, "cores": workers,
            "kind": "oracle",
            "sample": f"FP64 oracle, {len(sample_all)} smallest instances of the mix "
                      f"({nodes_all} nodes) x {steps_cpu} steps, one process per core"}
        if c1 is not None:
            # the same run on the oracle: its time, and the GPU's fields against it
            from oracle import oracle
            sys.path.insert(0, os.path.join(ROOT, "tests"))
            from oracle_helpers import oracle_sim
            from paper_2508_16997_gb300 import workloads as wl
            oracle.build()
            osim = oracle_sim(wl.frm(64))
            t0 = time.perf_counter()
            osim.step(args.frm64_steps)
            dt_o = time.perf_counter() - t0
            ref = osim.fields()

            def rel(a, r):
                return float(np.linalg.norm(a - r) / np.linalg.norm(r))
            c1["oracle"] = {"value": 64 * 64 * args.frm64_steps / dt_o / 1e6, "unit": UNIT,
                            "cores": 1, "seconds": dt_o,
                            "gpu_vs_oracle_rel_l2": {"u": rel(c1_fields[1:3], ref[1:3]),
                                                     "A": rel(c1_fields[3:6], ref[3:6]),
                                                     "target": 1e-12}}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def bench_frm64(steps: int, stream):
    """The four-roll mill 64^2 as specified (beta 0.5, Wi 5, Re 0.01, Sc 1e5,
    Ma 1e-3, FP64), `steps` steps from rest: returns the timing of the run
    and its fields after `steps` steps.  The first run from rest gives the
    fields and warms the handle up (graph capture); the timed run continues
    the same handle for another `steps` steps of identical cost.  A grid this
    small is bound by launch latency, not by HBM."""
    import torch
    from paper_2508_16997_gb300 import lbve, workloads as wl
    sim = lbve.Simulation([wl.frm(64)], precision=lbve.LBVE_FP64)
    sim.step(steps)
    fields = sim.fields(0)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    out = {"workload": "four-roll mill 64^2, beta 0.5, Wi 5, Re 0.01, Sc 1e5, Ma 1e-3, FP64, "
                       f"{steps} steps from rest", "value": 64 * 64 * steps / (ms / 1e3) / 1e6,
           "unit": UNIT, "ms": ms, "us_per_step": ms * 1e3 / steps,
           "finite": not bool(sim.status()[0])}
    return out, fields


def bench_frm_large(steps: int, stream) -> dict:
    """The small configuration's four-roll mill (beta 0.5, Wi 5, Re 0.01,
    Sc 1e5, Ma 1e-3) on 2048^2 and 4096^2 grids, one instance per handle, in
    FP32 deviations and FP64: per-launch step-kernel time (lbve_profile) over
    `steps` ordinary steps after a warm-up, MLUPS, and the kernel against its
    bound (HBM for FP32, the FP64 pipe for FP64)."""
    import torch
    from paper_2508_16997_gb300 import lbve, workloads as wl
    peak, peak_kind = measured_peaks()
    out = {"workload": "four-roll mill N^2, beta 0.5, Wi 5, Re 0.01, Sc 1e5, Ma 1e-3, from rest",
           "steps": steps}
    for N in (2048, 4096):
        inst = wl.frm(N)
        row = {}
        for name, prec in (("fp32", lbve.LBVE_FP32_DEV), ("fp64", lbve.LBVE_FP64)):
            sim = lbve.Simulation([inst], precision=prec)
            sim.step(5)
            torch.cuda.synchronize()
            lbve.lbve_profile(sim.h, steps + 1)
            sim.step(steps + 1)  # steps ordinary launches, then the final one
            n, tot, lo, hi = lbve.lbve_profile_read(sim.h, prec)
            lbve.lbve_profile(sim.h, 0)
            kms = tot / max(n, 1)
            mlups = inst.n_nodes / (kms / 1e3) / 1e6
            r = {"kernel_ms": kms, "kernel_ms_min": lo, "kernel_ms_max": hi, "launches": n,
                 "MLUPS": mlups, "finite": not bool(sim.status()[0])}
            if prec == lbve.LBVE_FP32_DEV:
                b = inst.n_nodes * bytes_per_lu(inst, 4)
                r["roofline"] = {"bound": "hbm", "achieved": b / (kms / 1e3) / 1e9, "peak": peak,
                                 "unit": "GB/s", "frac": b / (kms / 1e3) / 1e9 / peak,
                                 "peak_kind": peak_kind, "algorithmic_bytes_per_launch": b}
            else:
                r["roofline"] = measured_fp64_pipe(mlups)
            row[name] = r
            del sim
            torch.cuda.empty_cache()
        out[str(N)] = row
    return out


def bench_cylinder(steps: int, stream) -> dict:
    """Flow past a cylinder, Sec. 4.3 set-up at R = 64: 30R x 4R channel,
    blockage 1/2, curved wall fractions, inlet column with the fully
    developed Oldroyd-B profile (mean U_c), outlet at density 1.  MLUPS of
    the masked + open-channel path in FP32 and FP64, the same open channel
    without the cylinder for the cost of the solid mask, and the drag
    coefficient C_d = F_x / (rho U_avg^2 R), U_avg = U_c, at the end of the
    timed start-up run (not a steady value)."""
    import copy
    import torch
    from paper_2508_16997_gb300 import lbve, workloads as wl
    inst = wl.cylinder_channel(64, Wi=0.5, open_x=True)
    empty = copy.copy(inst)
    empty.solid = None
    empty.wall_q = None
    fluid = int((inst.solid == 0).sum())
    Uc = wl.velocity_scale(inst.Ma)
    out = {"workload": f"cylinder R=64 in a {inst.nx}x{inst.ny} channel, inlet profile "
                       f"(mean U_c) and outlet at rho = 1, beta {inst.beta}, Wi {inst.Wi}, "
                       f"Re {inst.Re}, Ma {inst.Ma}, curved walls "
                       f"({len(inst.wall_links())} wall links)",
           "fluid_nodes": fluid, "steps": steps}

    def timed(sim, n):
        sim.step(20)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.step(n)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    for prec, name, n in ((lbve.LBVE_FP32_DEV, "fp32", steps), (lbve.LBVE_FP64, "fp64",
                                                                max(1, steps // 10))):
        sim = lbve.Simulation([inst], precision=prec)
        ms = timed(sim, n)
        ref = lbve.Simulation([empty], precision=prec)
        ms_empty = timed(ref, n)
        tot = sim.totals(0)
        out[name] = {"MLUPS": fluid / ms / 1e3, "ms_per_step": ms,
                     "ms_per_step_without_cylinder": ms_empty,
                     "mask_overhead": ms / ms_empty - 1.0,
                     "drag_x": float(tot[12]),
                     "Cd_start_up": float(tot[12]) / (Uc * Uc * 64.0),
                     "note": "from rest: the drag stays 0 until the inlet's pressure wave "
                             "reaches the cylinder (~960/c_s = 1660 steps)",
                     "time_steps": int(sim.time(0)),
                     "finite": bool((sim.status() == 0).all())}
        del sim, ref
    return out


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
