"""Multi-rank host logic of bench.py on the CPU (gloo, world size 2).

The batched transform shards by batch with no data-path collective, so the
N-GPU benchmark runs one replica of the workload per rank; the only
collective is the timing reduction (slowest rank) and the barriers around
the timed region.  This runs those pieces as two gloo processes."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="env://")
    r, w, lr = bench.dist_env()
    dist.barrier()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, "cpu")
    fl = bench.flops_per_step(10, 12, 20)
    out[rank] = (r, w, lr, ms_max, bench.job_throughput(fl, w, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_slowest():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    import bench
    fl = bench.flops_per_step(10, 12, 20)
    for rank in range(world):
        r, w, lr, ms_max, gf = res[rank]
        assert (r, w, lr) == (rank, world, rank)
        assert ms_max == pytest.approx(15.0)
        assert gf == pytest.approx(world * fl / 15e-3 / 1e9)
