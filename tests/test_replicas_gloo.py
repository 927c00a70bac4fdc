"""The multi-rank (replica) timing path of bench.py on CPU with gloo, world_size 2.

The Magnus path does not shard (each Leja matvec needs the whole state), so N GPUs run N
independent replicas; the only cross-rank step is the max of the timed region and the whole-job
rate derived from it.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank          # rank 1 is the slow one
    ms = bench.max_over_ranks(ms_local)
    out[rank] = (ms, bench.replica_rate(40, ms, world))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_replica_rate():
    world, port = 2, _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        ms, rate = out[rank]
        assert ms == 150.0
        assert abs(rate - 2 * 40 / 0.150) < 1e-9


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_rate(100, 500.0, 1) == 200.0
