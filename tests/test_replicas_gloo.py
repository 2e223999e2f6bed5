"""Host-side logic of the multi-GPU (N > 1) bench path on CPU: world_size-2
gloo ranks.  On more GPUs the path runs independent seeded replicas (the
visibilities partition; no data-path collective), so what needs checking is
the job-level aggregation (max of the ranks' timed regions, sum of their
visibilities) and that the replicas draw different data of the same shape."""
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
    from paper_2206_15117_gb300 import synthetic as sy
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, nvis = bench.aggregate(100.0 + 50.0 * rank, 1000 + rank, dist)
    ob = sy.observation(3, time_samples=20, seed=sy.BASE_SEED + 3 + 1000 * rank)
    out[rank] = (ms, nvis, ob.nvis, float(ob.uvw[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_aggregation_and_replica_seeding():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    (ms0, n0, v0, u0), (ms1, n1, v1, u1) = out[0], out[1]
    assert ms0 == ms1 == 150.0            # the slowest rank's time, on every rank
    assert n0 == n1 == 2001               # visibilities of both ranks
    assert u0 != u1                       # different seeded replicas
    assert abs(v0 - v1) < 0.5 * max(v0, v1)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.aggregate(12.5, 77) == (12.5, 77)
