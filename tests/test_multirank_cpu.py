"""The bench's multi-GPU path (replicas, max over ranks) with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank measured its own step and iteration times; the slowest one decides
    mine = [10.0 + rank, 5.0 * (world - rank)]
    got = bench.max_over_ranks(mine, "cpu")
    rate = bench.whole_job_rate(1000.0, world, got[1] * 1e-3)
    dist.barrier()
    out.put((rank, got, rate, bench.env_rank()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_whole_job_rate(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, got, rate, env in res:
        assert got == [10.0 + world - 1, 5.0 * world]
        assert rate == pytest.approx(1000.0 * world / (5.0 * world * 1e-3))
        assert env == (rank, 0, world)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
