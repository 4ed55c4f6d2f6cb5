"""Multi-replica aggregation of bench.py on CPU ranks (gloo, world size 2).

The method does not shard across GPUs: N GPUs run N independent replicas
and the job's throughput is all ranks' units over the slowest rank's time.
These tests run that reduction over a real process group on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 180.0][rank]  # rank 1 is the slow one
    value, mx = bench.replica_throughput(1000.0, ms, world, device="cpu")
    out[rank] = (value, mx, bench.max_over_ranks(rank + 0.5, world, device="cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        value, mx, top = res[rank]
        assert mx == 180.0
        assert value == pytest.approx(2 * 1000.0 / 0.180)
        assert top == 1.5


def test_single_rank_needs_no_group():
    import bench
    value, ms = bench.replica_throughput(500.0, 250.0, 1)
    assert ms == 250.0 and value == pytest.approx(2000.0)
