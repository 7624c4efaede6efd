"""The multi-rank path of bench.py on CPU: two gloo ranks run independent,
differently seeded batches (weak scaling, no data exchange), the timing is
the maximum over ranks, and the reported value covers the work of all
ranks."""
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
        # a fake per-rank time: the slower rank must set the job's time
        t_local = 1.0 + rank
        t_max = bench.reduce_max(t_local, world)
        import torch
        ten = torch.tensor([nodes], dtype=torch.int64)
        gathered = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(gathered, ten)
        job_nodes = int(bench.reduce_sum(float(nodes), world))
        out[rank] = (nodes, t_max, [int(g.item()) for g in gathered],
                     bench.job_value(job_nodes, 10, t_max), bench.rank_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_host_path():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn",
                       join=True)
    (n0, t0, g0, v0, s0), (n1, t1, g1, v1, s1) = out[0], out[1]
    assert t0 == t1 == 2.0                 # max over ranks
    assert s0 != s1                        # independent seeds per rank
    assert g0 == g1 == [n0, n1]            # both ranks see both batches
    # whole-job value: all ranks' updates over the slowest rank's time
    assert v0 == v1 == pytest.approx((n0 + n1) * 10 / 2.0 / 1e6)
