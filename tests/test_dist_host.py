"""The benchmark's multi-rank host logic on CPU with two gloo ranks: every
rank gets the slowest rank's timed total, the whole-job rate counts every
rank's units over that time, and only rank 0 of the reference arm does work
(the others return without touching the oracle)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        r, w, local = bench.dist_env()
        dist.barrier()
        t = bench.max_over_ranks(10.0 * (rank + 1), w, "cpu")
        ref = bench.run_reference(None) if rank != 0 else "rank 0 skipped"
        q.put((r, w, local, t, bench.job_rate(100, w, t), ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[:3] for g in got] == [(0, 2, 0), (1, 2, 1)]
    for _, _, _, t, rate, _ in got:
        assert t == 20.0                       # the slower rank's total on both ranks
        assert rate == pytest.approx(2 * 100 / 0.020)
    assert got[1][5] is None                   # rank 1 of the reference arm: no work


def test_single_rank_is_its_own_total():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(4096, 1, 5.0) == pytest.approx(4096 / 0.005)
