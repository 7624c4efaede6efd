"""The multi-rank path of bench.py on CPU: two gloo ranks build independent,
differently seeded batches and plan their device workspaces through the
library's host-only lbve_workspace_bytes (weak scaling, no data exchange),
the timing is the maximum over ranks, and the reported value covers the work
of all ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        insts = bench.workload(rank, 6)
        nodes = sum(i.n_nodes for i in insts)
        ws = bench.workspace_bytes(insts)
        # a fake per-rank time: the slower rank must set the job's time
        t_local = 1.0 + rank
        t_max = bench.reduce_max(t_local, world)
        import torch
        ten = torch.tensor([nodes], dtype=torch.int64)
        gathered = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gathered, ten)
        job_nodes = int(bench.reduce_sum(float(nodes), world))
        wsg = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(wsg, torch.tensor([ws], dtype=torch.int64))
        out[rank] = (nodes, t_max, [int(g.item()) for g in gathered],
                     bench.job_value(job_nodes, 10, t_max), bench.rank_seed(rank),
                     [int(g.item()) for g in wsg])
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_host_path():
    import bench
    from paper_2508_16997_gb300 import build
    build.build()
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn",
                       join=True)
    (n0, t0, g0, v0, s0, w0), (n1, t1, g1, v1, s1, w1) = out[0], out[1]
    assert t0 == t1 == 2.0                 # max over ranks
    assert s0 != s1                        # independent seeds per rank
    assert g0 == g1 == [n0, n1]            # both ranks see both batches
    # whole-job value: all ranks' updates over the slowest rank's time
    assert v0 == v1 == pytest.approx((n0 + n1) * 10 / 2.0 / 1e6)
    # each rank planned its own batch: the same plan as this process makes for
    # that rank's seed, at least the two 36-plane float32 population buffers
    assert w0 == w1
    for r, n in ((0, n0), (1, n1)):
        assert w0[r] == bench.workspace_bytes(bench.workload(r, 6))
        assert w0[r] >= 2 * 36 * 4 * n
    assert w0[0] != w0[1]
