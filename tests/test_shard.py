"""Host logic of the multi-GPU batched path (paper_2605_24840_gb300.shard):
the LPT partition of independent problems over ranks and the host gather of
their reports, with world_size 2 over gloo on the CPU (no GPU, no collective
in the data path)."""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_2605_24840_gb300 import shard


def test_lpt_partition_is_a_deterministic_cover():
    rng = np.random.default_rng(3)
    costs = rng.uniform(1, 100, 57).tolist()
    for m in (1, 2, 3, 8):
        parts = shard.lpt_partition(costs, m)
        assert parts == shard.lpt_partition(costs, m)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        assert all(p == sorted(p) for p in parts)


@pytest.mark.parametrize("seed", range(20))
def test_lpt_partition_within_grahams_bound_of_the_optimum(seed):
    # brute force over all assignments of <= 8 items to 2 or 3 ranks
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 9))
    m = int(rng.integers(2, 4))
    costs = rng.uniform(1, 50, n).tolist()
    parts = shard.lpt_partition(costs, m)
    lpt = max(sum(costs[i] for i in p) for p in parts)
    opt = min(max(sum(c for c, r in zip(costs, a) if r == k) for k in range(m))
              for a in itertools.product(range(m), repeat=n))
    assert lpt <= (4.0 / 3.0 - 1.0 / (3.0 * m)) * opt + 1e-9


def test_ns_cost_grows_with_order_and_with_a_smaller_margin():
    assert shard.ns_cost(512) > shard.ns_cost(256)
    assert shard.ns_cost(256, 1e-3) > shard.ns_cost(256, 1e-1)


def test_run_sharded_single_rank():
    mine, res = shard.run_sharded(5, [1, 2, 3, 4, 5], lambda idx: [i * i for i in idx], 0, 1)
    assert mine == [0, 1, 2, 3, 4] and res == [0, 1, 4, 9, 16]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        def gather(obj):
            out = [None] * world
            dist.all_gather_object(out, obj)
            return out

        computed = []

        def compute(idx):
            computed.extend(idx)
            return [{"item": i, "value": 3 * i + 1, "rank": rank} for i in idx]

        mine, res = shard.run_sharded(len(costs), costs, compute, rank, world, gather)
        q.put((rank, mine, sorted(computed), res))
    finally:
        dist.destroy_process_group()


def test_run_sharded_world_size_two_over_gloo():
    import torch.multiprocessing as mp
    costs = [float(d) ** 3 for d in (32, 512, 64, 448, 96, 384, 128, 320, 160, 288, 192, 256)]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    parts = shard.lpt_partition(costs, world)
    for rank, mine, computed, res in got:
        assert mine == parts[rank] and computed == parts[rank]  # each rank solved only its share
        assert [r["value"] for r in res] == [3 * i + 1 for i in range(len(costs))]  # every report gathered
        assert all(r["rank"] == next(k for k in range(world) if r["item"] in parts[k]) for r in res)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert max(loads) / min(loads) < 1.3
