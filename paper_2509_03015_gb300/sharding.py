"""Multi-process sharding of independent systems (one process per GPU).

The batched workload is a set of independent instances: ranks take disjoint
subsets, balanced by work (N_k n_k^3), with no collective on the data path;
only the timing is reduced (max over ranks).  Pure host logic."""
from __future__ import annotations


def instance_work(N: int, n: int) -> float:
    return float(N) * n ** 3


def shard_instances(shapes, world: int):
    """Greedy longest-processing-time assignment of instances (N_k, n_k) to
    `world` ranks.  Returns a list of index lists, one per rank, each sorted."""
    order = sorted(range(len(shapes)), key=lambda k: -instance_work(*shapes[k]))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += instance_work(*shapes[k])
    return [sorted(x) for x in out]


def rank_share(shapes, rank: int, world: int):
    return shard_instances(shapes, world)[rank]
