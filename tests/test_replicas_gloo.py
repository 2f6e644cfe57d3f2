"""Host-side logic of the multi-GPU benchmark (independent replicas): the slowest
rank's time and the whole-job rate, over a world-size-2 gloo process group on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 2.0 + rank  # rank 1 is the slowest
        m = bench.max_over_ranks(dist, t)
        q.put((rank, m, bench.job_rate(world, 1000.0, m)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in out:
        assert m == 3.0
        assert rate == pytest.approx(2 * 1000.0 / 3.0)


def test_single_process_identity():
    import bench

    assert bench.max_over_ranks(None, 1.5) == 1.5
    assert bench.job_rate(1, 10.0, 2.0) == 5.0
