"""The replicated multi-GPU bench path on CPU: two gloo ranks, each with its own vehicle
(replicas, no collective on the data path); the whole-job figures are the slowest rank's time
and the sum of the ranks' points."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev_s, pts = (1.5, 1000.0) if rank == 0 else (2.5, 3000.0)
    t, p = bench.aggregate_ranks(dev_s, pts, world, "cpu")
    veh = bench.Vehicle(rank)
    out.put((rank, t, p, float(veh.seq.s0)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_summed_points():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]
    assert [r[2] for r in res] == [4000.0, 4000.0]
    assert res[0][3] != res[1][3]        # each rank drives its own vehicle
