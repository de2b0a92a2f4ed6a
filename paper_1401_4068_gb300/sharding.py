"""Assignment of a workload's estimates to ranks (one process per GPU).

Estimates are independent, so the path shards without any data exchange. The unit of
assignment is a group: all estimates that share (series, analysis start, window) — the original
and its surrogates — so that a rank can form every p-value of its groups on its own. Groups are
placed largest-first on the least-loaded rank (cost = N^2 * D summed over the group), which is
deterministic for a given workload and world size. Host-only logic; no GPU involved.
"""
from __future__ import annotations

from collections import OrderedDict
from typing import Dict, List, Sequence, Tuple


def groups(instances: Sequence, n_points, joint_dim) -> "OrderedDict[Tuple[int, int, int], List[int]]":
    """Instance indices grouped by (series, t_start, window), in first-appearance order."""
    g: "OrderedDict[Tuple[int, int, int], List[int]]" = OrderedDict()
    for i, it in enumerate(instances):
        g.setdefault((int(it.series), int(it.t_start), int(it.window)), []).append(i)
    return g


def shard(workload, world_size: int) -> List[List[int]]:
    """Instance indices per rank (each list in increasing order)."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    gs = groups(workload.instances, workload.n_points, workload.joint_dim)
    costed = []
    for key, idx in gs.items():
        c = sum(workload.n_points(workload.instances[i]) ** 2 * workload.joint_dim(workload.instances[i])
                for i in idx)
        costed.append((c, key, idx))
    costed.sort(key=lambda x: (-x[0], x[1]))
    load = [0] * world_size
    out: List[List[int]] = [[] for _ in range(world_size)]
    for c, _, idx in costed:
        r = min(range(world_size), key=lambda k: (load[k], k))
        load[r] += c
        out[r].extend(idx)
    return [sorted(x) for x in out]


def rank_load(workload, parts: List[List[int]]) -> List[int]:
    return [sum(workload.n_points(workload.instances[i]) ** 2 * workload.joint_dim(workload.instances[i])
                for i in p) for p in parts]
