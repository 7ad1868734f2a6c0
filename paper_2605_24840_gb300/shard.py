"""Host-side sharding of a batch of independent reflector problems over ranks.

Independent matrices need no exchange: each rank takes a fixed share of the
batch (longest-processing-time-first on the per-matrix cost d^3 times the
step count predicted from the margin), solves it with the batched call on its
own GPU, and the per-matrix reports are gathered on the host.  The only
collective is that host gather (torch.distributed all_gather_object over any
backend); the matrices themselves never leave their rank.
"""
from __future__ import annotations

import heapq
import math


def ns_cost(d: int, delta_rel: float | None = None) -> float:
    """Work estimate of one problem: d^3 per Newton-Schulz step times the
    number of steps ~ log_1.5(1/gamma) + 6 (gamma = relative margin, 1e-2
    when unknown)."""
    g = delta_rel if (delta_rel is not None and delta_rel > 0.0) else 1e-2
    g = min(max(g, 1e-12), 1.0)
    steps = math.log(1.0 / g) / math.log(1.5) + 6.0
    return float(d) ** 3 * steps


def lpt_partition(costs, n_ranks: int):
    """Greedy longest-processing-time-first assignment of items (by cost) to
    n_ranks bins: items in decreasing cost (ties by index), each to the bin
    with the least load (ties by rank).  Deterministic, so every rank computes
    the same partition.  Returns a list of index lists, each ascending."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(n_ranks)]
    heapq.heapify(heap)
    parts = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def run_sharded(n_items: int, costs, compute, rank: int, world_size: int, gather=None):
    """Run `compute(indices) -> list of per-item results` on this rank's share
    of the LPT partition and gather every rank's results on the host.

    gather: a function (object) -> list of objects, one per rank (for example
    torch.distributed.all_gather_object wrapped to return the list); None
    with world_size == 1.  Returns (my_indices, results) with results[i] the
    result of item i from whichever rank computed it."""
    if len(costs) != n_items:
        raise ValueError("one cost per item")
    parts = lpt_partition(costs, world_size)
    mine = parts[rank]
    local = compute(mine)
    if len(local) != len(mine):
        raise ValueError("compute must return one result per index")
    if world_size == 1:
        gathered = [list(zip(mine, local))]
    else:
        if gather is None:
            raise ValueError("a gather function is needed for world_size > 1")
        gathered = gather(list(zip(mine, local)))
    results = [None] * n_items
    for part in gathered:
        for i, res in part:
            results[i] = res
    return mine, results


def reflectors_sharded(Hs, ks, ss, tol, policy, rank, world_size, gather=None, options=None, costs=None):
    """Batched reflectors over ranks: this rank solves its LPT share with
    rsign_reflector_batched_ex on its current GPU and keeps its R matrices;
    the reports (rsign_info as dicts) of all items are gathered.
    Returns (my_indices, my_outputs, reports)."""
    from . import reflector_batched  # the C ABI binding (fails loudly without the library)

    n = len(Hs)
    if costs is None:
        costs = [ns_cost(int(H.shape[0])) for H in Hs]
    outs_mine = {}

    def compute(idx):
        if not idx:
            return []
        outs, infos, _ = reflector_batched([Hs[i] for i in idx], [ks[i] for i in idx], [ss[i] for i in idx],
                                           tol=tol, policy=policy, options=options)
        for j, i in enumerate(idx):
            outs_mine[i] = outs[j]
        return [info.as_dict() for info in infos]

    mine, reports = run_sharded(n, costs, compute, rank, world_size, gather)
    return mine, [outs_mine[i] for i in mine], reports
