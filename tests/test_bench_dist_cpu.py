"""The benchmark's multi-rank path (replicas, one per GPU) on CPU: two gloo
ranks reduce their step times to the slowest one and report the whole-job
value; rank 0 alone prints."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 100.0 + 50.0 * rank           # rank 1 is the slowest
        ms_max = bench.max_over_ranks(world, ms)
        value = bench.whole_job_value(2.0e12, world, ms_max)
        dist.barrier()
        q.put((rank, ms_max, value))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_whole_job_value(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms_max, value in res:
        assert ms_max == 150.0
        # 2 ranks x 2e12 flops over 150 ms = 26.67 TFLOP/s
        assert abs(value - 2 * 2.0e12 / 0.150 / 1e12) < 1e-9


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(1, 3.5) == 3.5
    assert abs(bench.whole_job_value(1.0e12, 1, 1000.0) - 1.0) < 1e-12
