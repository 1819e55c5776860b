"""CPU: the multi-rank path of bench.py (independent replicas, one per rank) with
two gloo ranks: the job time is the slowest rank's, the job throughput counts
every rank's work, and only rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.env_rank()
    seconds = [2.0, 3.0][rank]  # rank 1 is the slower replica
    t = bench.max_over_ranks(seconds, dist, "cpu")
    value = bench.job_throughput(w, 100.0, t)
    out.put((r, w, local, t, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    # every rank sees the slowest rank's time and the same whole-job throughput
    assert all(r[3] == 3.0 for r in res)
    assert all(r[4] == pytest.approx(2 * 100.0 / 3.0) for r in res)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.5, None, "cpu") == 1.5
    assert bench.job_throughput(1, 10.0, 2.0) == 5.0
