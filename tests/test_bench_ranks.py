"""Multi-process path of bench.py on the CPU: with N ranks the ranks split
one network (or run replicas on request) and the reported value is all
ranks' events over the slowest rank's time.  Two gloo ranks check the
reduction and the barrier."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier()
    ms = 10.0 + 5.0 * rank          # rank 1 is the slowest
    events = 1000 * (rank + 1)
    res = bench.reduce_over_ranks(ms, events, extra=float(rank))
    out[rank] = res
    dist.destroy_process_group()


def test_two_rank_reduction_max_time_sum_events():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (15.0, 3000, 1.0)


def test_single_process_reduction_is_identity():
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks(12.5, 77, 3.0) == (12.5, 77, 3.0)


def test_several_ranks_partition_one_network_by_default():
    import bench
    up = bench.use_partition
    assert up("balanced-112500-fp32", "simulate", 4, False, False)
    assert not up("balanced-112500-fp32", "simulate", 4, False, True)
    assert not up("balanced-112500-fp32", "simulate", 1, False, False)
    assert up("balanced-112500-fp32", "simulate", 1, True, False)
    assert not up("balanced-112500-stdp-bf16", "simulate", 4, False, False)
    assert not up("deliver-112500-fp32", "deliver", 8, False, False)
    with pytest.raises(SystemExit):
        up("deliver-112500-fp32", "deliver", 1, True, False)
