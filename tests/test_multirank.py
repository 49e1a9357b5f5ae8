"""The multi-process benchmark path on CPU: two gloo ranks run replicas and the
whole-job numbers are the slowest rank's time and the sum of the work."""
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


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" 10 + r ms and did 1000 * (r + 1) voxel-iterations
    t, v = bench.reduce_over_ranks(dist, 10.0 + rank, 1000 * (rank + 1), "cpu")
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_reduction_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 10.0 + (world - 1)          # max over ranks
        assert v == sum(1000 * (r + 1) for r in range(world))
