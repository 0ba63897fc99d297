"""The N > 1 path of bench.py on CPU: two gloo ranks. The benchmark runs independent replicas
(one cavity per GPU, no data-path collective); only the job time is reduced across ranks (max)
and the value is all ranks' updates over the slowest rank's time. The reference arm runs and
prints on rank 0 only."""
import contextlib
import io
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        slowest = bench.max_over_ranks(1.5 + rank, dist, "cpu")
        rate = bench.whole_job_rate(256 * 256 * 1000, world, slowest)
        # the reference arm prints only on rank 0; other ranks return without work
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            if rank != 0:
                bench.reference_arm(None, world, rank)
        q.put((rank, slowest, rate, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_bench():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, printed in res:
        assert slowest == 2.5  # the slower rank's time on every rank
        assert rate == pytest.approx(256 * 256 * 1000 * 2 / 2.5 / 1e6)
        if rank == 1:
            assert printed == ""


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.whole_job_rate(1e6, 1, 2.0) == pytest.approx(0.5)


def test_step_launch_count_follows_the_graph_decomposition():
    """bench.py's gpu_launches: mclbm_step(n) launches n step kernels plus one epoch kernel per
    captured graph of 2^k steps (k = 1..10, largest first)."""
    import bench
    assert bench.step_launches(0) == 0
    assert bench.step_launches(1) == 1
    assert bench.step_launches(2) == 3
    assert bench.step_launches(64) == 65
    assert bench.step_launches(1000) == 1000 + 6   # 512 + 256 + 128 + 64 + 32 + 8
    assert bench.step_launches(1001) == 1001 + 6
    assert bench.step_launches(3000) == 3000 + 8   # 1024 + 1024 + 512 + 256 + 128 + 32 + 16 + 8
