"""The multi-GPU form of the benchmark is replicas only (one independent
copy of the workload per rank, no collective on the data path): the
cross-rank aggregation (max-over-ranks time, whole-job rate) with two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "processed" 1000 cell-iterations in 10 (r + 1) ms
    rate, ms = bench.replicas_value(dist, world, 1000, 10.0 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, ms))


def test_replicas_take_the_slowest_rank():
    world = 2
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms in out:
        assert ms == 20.0                      # the slower rank's time
        assert abs(rate - 2 * 1000 / 20e-3 / 1e6) < 1e-12   # both ranks' work over it


def test_single_rank_rate():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms = bench.replicas_value(None, 1, 491520 * 65, 40.0, "cpu")
    assert ms == 40.0 and abs(rate - 491520 * 65 / 40e-3 / 1e6) < 1e-9
