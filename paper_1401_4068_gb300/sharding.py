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


# ---------------------------------------------------------------------------------------
# Sharded runs: each rank computes a cost-balanced share of a workload's units (analysis time
# points of a surrogate test or delay scan, each with all of its estimates; or the groups of a
# te_estimate batch), writes one row of results per unit, and all ranks gather the rows into the
# full result in unit order. The only exchange is this gather of a few doubles per unit, after
# the compute: no collective on the data path.
# ---------------------------------------------------------------------------------------
def balance(costs: Sequence[float], world_size: int) -> List[List[int]]:
    """Unit indices per rank: largest cost first onto the least-loaded rank (ties to the lower
    rank), each list in increasing order. Deterministic for given costs and world size."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(costs)), key=lambda u: (-costs[u], u))
    load = [0.0] * world_size
    out: List[List[int]] = [[] for _ in range(world_size)]
    for u in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        load[r] += costs[u]
        out[r].append(u)
    return [sorted(x) for x in out]


def time_point_costs(workload) -> List[float]:
    """Cost of each analysis start of a one-series surrogate or delay-scan workload: N^2 D summed
    over the estimates of that start (every start has 1 + S estimates per scanned delay)."""
    s = workload.series[0]
    per = []
    for t in workload.t_starts[0]:
        n = s.R * workload.window
        per.append(float(n) * n * (1 + 2 * s.d) * (workload.S + 1))
    return per


def gather_rows(rows, parts: List[List[int]], n_units: int, group=None):
    """All-gather of per-rank result rows: `rows` is this rank's float64 tensor [len(parts[rank]),
    width] (row i belongs to unit parts[rank][i]); returns the [n_units, width] tensor in unit
    order on every rank. Works with any torch.distributed backend (NCCL for device tensors, gloo
    for host tensors)."""
    import torch
    import torch.distributed as dist
    ws = len(parts)
    width = rows.shape[1]
    m = max(len(p) for p in parts)
    pad = torch.zeros((m, width), dtype=rows.dtype, device=rows.device)
    pad[: rows.shape[0]] = rows
    bufs = [torch.empty_like(pad) for _ in range(ws)]
    dist.all_gather(bufs, pad, group=group)
    full = torch.empty((n_units, width), dtype=rows.dtype, device=rows.device)
    for r, p in enumerate(parts):
        if p:
            idx = torch.tensor(p, dtype=torch.long, device=rows.device)
            full[idx] = bufs[r][: len(p)]
    return full
