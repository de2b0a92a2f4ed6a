"""Multi-rank host logic on the CPU: the instance-to-rank assignment covers every estimate once,
keeps each original with its surrogates, balances cost, and a 2-rank gloo run that computes its
shard (with the oracle) and gathers the results reproduces the single-process answer."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import sharding


def _small_surrogate_workload():
    w = I.config(1)
    s = w.series[0]
    s.perms = I.permutations(np.random.default_rng(3), 5, s.R)
    insts = [I.Instance(0, t, 5, p) for t in (40, 120, 200) for p in [-1] + list(range(5))]
    return I.Workload("sharding test", [s], insts, k=4, t_starts=[[40, 120, 200]], window=5, S=5)


@pytest.mark.parametrize("ws", [1, 2, 3, 8])
def test_shards_cover_every_estimate_once(ws):
    w = I.config(4, n_pairs=6, n_t=5)
    parts = sharding.shard(w, ws)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(w.instances)))
    load = sharding.rank_load(w, parts)
    biggest = max(w.n_points(i) ** 2 * w.joint_dim(i) for i in w.instances)
    assert max(load) - min(load) <= biggest


def test_groups_stay_on_one_rank():
    w = _small_surrogate_workload()
    parts = sharding.shard(w, 2)
    for p in parts:
        keys = {(w.instances[i].series, w.instances[i].t_start) for i in p}
        for key in keys:
            members = [i for i, it in enumerate(w.instances) if (it.series, it.t_start) == key]
            assert set(members) <= set(p)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w = _small_surrogate_workload()
    mine = sharding.shard(w, ws)[rank]
    te = oracle.te_batch(w.series, [w.instances[i] for i in mine], w.k, n_threads=1)
    got = [None] * ws
    dist.all_gather_object(got, (mine, te.tolist()))
    if rank == 0:
        full = np.full(len(w.instances), np.nan)
        for idx, vals in got:
            full[idx] = vals
        q.put(full.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_run_matches_single_process():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    full = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _small_surrogate_workload()
    ref = oracle.te_batch(w.series, w.instances, w.k)
    np.testing.assert_array_equal(np.array(full), ref)


def _oracle_rows(w, t_list):
    """Rows (te_orig, p, te_surr[S]) of a surrogate test at the listed starts, by the oracle."""
    import oracle
    rows = []
    for t in t_list:
        insts = [I.Instance(0, t, w.window, p) for p in range(-1, w.S)]
        v = oracle.te_batch(w.series, insts, w.k, n_threads=1)
        rows.append([v[0], oracle.pvalue(v[0], v[1:]), *v[1:]])
    return np.array(rows, dtype=np.float64).reshape(len(t_list), 2 + w.S)


def _rows_worker(rank, ws, port, q):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w = _small_surrogate_workload()
    parts = sharding.balance(sharding.time_point_costs(w), ws)
    mine = _oracle_rows(w, [w.t_starts[0][u] for u in parts[rank]])
    full = sharding.gather_rows(torch.from_numpy(mine), parts, len(w.t_starts[0]))
    q.put((rank, parts, full.numpy().tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_surrogate_test_rows_match_single_process():
    """The bench's sharded path: analysis starts balanced over 2 gloo ranks, each rank's rows
    (original TE, p-value, surrogate TEs) all-gathered into start order on every rank, equal to
    one process computing all starts."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rows_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=240) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = _small_surrogate_workload()
    ref = _oracle_rows(w, w.t_starts[0])
    for rank, parts, full in got:
        assert sorted(u for p in parts for u in p) == list(range(len(w.t_starts[0])))
        assert all(parts)  # every rank has work
        np.testing.assert_array_equal(np.array(full), ref)


@pytest.mark.parametrize("ws", [1, 2, 3, 8])
def test_balance_covers_units_once_and_balances(ws):
    rng = np.random.default_rng(ws)
    costs = list(rng.integers(1, 100, 37).astype(float))
    parts = sharding.balance(costs, ws)
    assert sorted(u for p in parts for u in p) == list(range(37))
    load = [sum(costs[u] for u in p) for p in parts]
    assert max(load) - min(load) <= max(costs)
    assert parts == sharding.balance(costs, ws)  # deterministic
