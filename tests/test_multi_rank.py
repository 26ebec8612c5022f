"""The N > 1 path of bench.py on CPU: two gloo ranks (the GPU launch uses
NCCL with one process per GPU; the host logic is the same).  Replicas only:
each rank runs an independent pore with its own seed and the timing is the
maximum over ranks.  No GPU is touched."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank, world)
    wl = bench.workload_for("pore", rank)
    bench.barrier(world)
    q.put((rank, t, wl.seed, wl.n_nodes))
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, s0, n0), (r1, t1, s1, n1) = out
    assert t0 == t1 == 2.5          # every rank sees the slowest rank's time
    assert s0 != s1 and n0 == n1    # independent replicas of the same workload
