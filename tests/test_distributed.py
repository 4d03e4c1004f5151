"""The N > 1 path of bench.py on CPU: world_size-2 gloo process group.

bench.py runs one independent replica per rank (no data-path collective);
the job time is the maximum over ranks and the job throughput the sum of the
replicas' work.  This checks those two steps across real processes.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank * 0.5, dist, "cpu")
    rate = bench.job_throughput(3.0, t, world)
    dist.barrier()
    out[rank] = (t, rate)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput_gloo_world2():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        t, rate = res[rank]
        assert t == 1.5               # the slowest rank's time on every rank
        assert rate == world * 3.0 / 1.5


def test_single_process_defaults():
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_throughput(64, 2.0, 1) == 32.0
