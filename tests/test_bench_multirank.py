"""The benchmark's multi-rank logic on two gloo ranks (CPU): every rank ends up
with the slowest rank's time, the whole-job rate counts every rank's steps, and
each replica decomposes its own tensor (same shapes, its own data seed)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, queue):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.slowest_rank_ms(times[rank], dist, "cpu")
        rate = bench.job_rate(5, world, ms)
        w = bench.replica_workload(bench.WORKLOADS["lowrank100_rhosvd"], rank)
        queue.put((rank, ms, rate, w.seed, w.dims))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time():
    world, times = 2, [12.5, 40.0]
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, queue)) for r in range(world)]
    for p in procs:
        p.start()
    results = [queue.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort()
    import bench
    base = bench.WORKLOADS["lowrank100_rhosvd"]
    for rank, ms, rate, seed, dims in results:
        assert ms == max(times)                                  # every rank sees the slowest time
        assert rate == pytest.approx(world * 5 / (max(times) / 1e3))
        assert seed == base.seed + rank and dims == base.dims    # own data, same shapes
    assert results[0][3] != results[1][3]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.slowest_rank_ms(7.0) == 7.0
    assert bench.job_rate(10, 1, 500.0) == pytest.approx(20.0)
    w = bench.WORKLOADS["decay512_rsthosvd"]
    assert bench.replica_workload(w, 0) == w
