"""The replicas path of bench.py at world size 2 (gloo, CPU): every rank gets
the slowest rank's elapsed time and the whole-job per-reflector value."""
import os
import socket


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [300.0, 420.0][rank]  # this rank's own K-step time, ms
        m = bench.max_over_ranks(torch, elapsed, world)
        q.put((rank, m, bench.job_ms_per_unit(m, 3, world)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [420.0, 420.0]
    assert all(abs(g[2] - 420.0 / 6) < 1e-12 for g in got)


def test_single_rank_is_the_identity():
    import torch
    import bench
    assert bench.max_over_ranks(torch, 12.5, 1) == 12.5
    assert bench.job_ms_per_unit(12.5, 5, 1) == 2.5
