"""Host logic of the N-rank benchmark (independent replicas, one per GPU): the
job time is the slowest rank's and the rate counts every rank's work; under
torchrun the reference arm runs on rank 0 only.  Checked with two gloo ranks
on the CPU."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    t = bench.job_time_ms(10.0 + 5.0 * rank, world, torch.device("cpu"))
    r = bench.job_rate(1000, world, t)

    class Args:
        workload, steps, warmup = "turbulent3d-256", 1, 1

    rc = bench.run_reference(Args) if rank == 1 else None
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, r, rc))


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, t, r, rc = q.get(timeout=180)
            out[rank] = (t, r, rc)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert set(out) == {0, 1}
    for rank in (0, 1):
        assert out[rank][0] == 15.0
        assert out[rank][1] == pytest.approx(1000 * 2 / 0.015)
    assert out[1][2] == 0  # the reference arm does no work off rank 0
