"""Multi-rank host logic of bench.py on CPU with gloo (world size 2): each rank
draws its own replica of the workload, the job time is the slowest rank's,
and the whole-job rate counts every rank's pixel-solves."""
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


def _worker(rank, world, port, q):
    import sys
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_1509_06004_b300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = bench.WORKLOADS["single-64x64"](bench.rank_seed(0, rank))
    local_t = 1.0 + rank                     # rank 1 is the slow one
    t = bench.max_over_ranks(local_t, world, None)
    dist.barrier()
    q.put((rank, t, int(wl.images[0].w_h.sum()), wl.pixel_solves))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == out[1][1] == 2.0          # max over ranks
    assert out[0][2] != out[1][2]                 # different replicas
    rate = world * out[0][3] / out[0][1]          # whole-job pixel-solves/s
    assert rate == pytest.approx(4096.0)
