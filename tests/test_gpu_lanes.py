"""One estimate per lane (the lane kernel, forced here with te.SHARE_LANES; by default it takes
groups of at least 32 estimates with d >= 3): a group of at least 8 estimates that share y_t and y-
(the original and its trial-shuffled surrogates, every scanned delay u) runs with a warp per
query point and one estimate per lane; a reference whose target-part distance already reaches
every lane's radius is skipped for all of them. Per-point radii and counts must equal the
unshared search and the CPU oracle bit for bit, TE within 1e-6 nats of the oracle: every d the
kernel takes (2..8), ragged groups (8, 9, 31, 32, 33, 70 estimates), point counts below, at and
above one 32-point chunk, k = 1..4, many equal distances, delay scans, mixed batches, a bad
permutation entry, determinism."""
import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _run(h, ds, insts, k, mode):
    te.te_set_sharing(h, mode)
    try:
        res = te.te_estimate(h, ds, insts, k, want_err=True, want_counts=True)
        torch.cuda.synchronize()
        te.te_sync_status(h)
        paths = te.te_last_paths(h)
        ops, _ = te.te_last_alu_ops(h)
        pairs, alg, swept = te.te_last_work(h)
    finally:
        te.te_set_sharing(h, te.SHARE_AUTO)
    return res, paths, ops, alg


def _series(rng, R, T, d, tau, u, S, ties=False):
    if ties:
        src = rng.integers(0, 4, (R, T)).astype(np.float32)
        tgt = rng.integers(0, 4, (R, T)).astype(np.float32)
    else:
        src, tgt = I.ar2_pair(rng, R, T)
    return I.Series(src, tgt, d=d, tau=tau, u=u, perms=I.permutations(rng, S, R))


def _check_against_unshared_and_oracle(h, series, insts, k, n_lane, oracle_idx=None):
    ds = te.to_device(series)
    off, p0, _, _ = _run(h, ds, insts, k, te.SHARE_NONE)
    on, p1, ops1, alg1 = _run(h, ds, insts, k, te.SHARE_LANES)
    assert p0[0] == 0 and p1[0] == n_lane
    assert ops1 < alg1
    assert torch.equal(off["counts"], on["counts"]) and torch.equal(off["eps"], on["eps"])
    diff = (off["te"] - on["te"]).abs()
    assert bool((diff <= off["err_bound"] + on["err_bound"]).all())
    sub = insts if oracle_idx is None else [insts[i] for i in oracle_idx]
    o_te, o_counts, o_eps = oracle.te_batch(series, sub, k, want_counts=True)
    if oracle_idx is None:
        np.testing.assert_array_equal(on["eps"].cpu().numpy(), o_eps)
        np.testing.assert_array_equal(on["counts"].cpu().numpy(), o_counts)
        got = on["te"].cpu().numpy()
    else:
        N = [series[it.series].R * it.window for it in insts]
        off_pt = np.concatenate([[0], np.cumsum(N)])
        eps = on["eps"].cpu().numpy()
        counts = on["counts"].cpu().numpy()
        o = 0
        for i in oracle_idx:
            n = N[i]
            np.testing.assert_array_equal(eps[off_pt[i]:off_pt[i] + n], o_eps[o:o + n])
            np.testing.assert_array_equal(counts[3 * off_pt[i]:3 * (off_pt[i] + n)], o_counts[3 * o:3 * (o + n)])
            o += n
        got = on["te"].cpu().numpy()[oracle_idx]
    assert np.max(np.abs(got - o_te)) <= TOL
    assert np.all(on["err_bound"].cpu().numpy() <= TOL)
    return on


@pytest.mark.parametrize("d", [2, 3, 4, 5, 6, 7, 8])
def test_every_dimension_equals_unshared_and_oracle(te_handle, d):
    rng = np.random.default_rng(300 + d)
    s = _series(rng, 41, 80, d, 1, 3, 11)
    t0 = 2 + (d - 1)
    insts = [I.Instance(0, t0 + 5, 3, p) for p in range(-1, 11)]  # 12 estimates of 123 points
    _check_against_unshared_and_oracle(te_handle, [s], insts, 4, 12)


@pytest.mark.parametrize("n_est", [8, 9, 31, 32, 33, 70])
def test_ragged_lane_blocks(te_handle, n_est):
    rng = np.random.default_rng(400 + n_est)
    s = _series(rng, 60, 60, 3, 2, 4, n_est - 1)
    insts = [I.Instance(0, 20, 2, p) for p in range(-1, n_est - 1)]
    idx = sorted({0, 1, n_est // 2, n_est - 1})
    _check_against_unshared_and_oracle(te_handle, [s], insts, 4, n_est, oracle_idx=idx)


@pytest.mark.parametrize("R,window,k", [(6, 3, 4), (8, 4, 1), (16, 2, 2), (11, 3, 3), (300, 3, 4), (700, 2, 4)])
def test_point_counts_around_one_chunk_and_every_k(te_handle, R, window, k):
    """N = 18 and 32 (one chunk, ragged or full), 33 (two), up to 1400 points; k = 1..4."""
    rng = np.random.default_rng(500 + R + k)
    s = _series(rng, R, 50, 2, 1, 2, 9)
    insts = [I.Instance(0, 10, window, p) for p in range(-1, 9)]
    idx = None if R * window <= 400 else [0, 3, 9]
    _check_against_unshared_and_oracle(te_handle, [s], insts, k, 10, oracle_idx=idx)


@pytest.mark.parametrize("d", [2, 5])
def test_many_equal_distances(te_handle, d):
    rng = np.random.default_rng(600 + d)
    s = _series(rng, 90, 40, d, 1, 2, 15, ties=True)
    insts = [I.Instance(0, 12, 3, p) for p in range(-1, 15)]
    _check_against_unshared_and_oracle(te_handle, [s], insts, 4, 16)


def test_mixed_batch_lanes_bundles_and_unshared(te_handle):
    """Two lane groups of different d, a small group in bundles (d = 3), single estimates
    unshared, in one call."""
    rng = np.random.default_rng(700)
    src, tgt = I.ar2_pair(rng, 50, 150)
    perms = I.permutations(rng, 12, 50)
    s2 = I.Series(src, tgt, d=2, tau=1, u=5, perms=perms)
    s3 = I.Series(src, tgt, d=3, tau=2, u=5, perms=perms)
    insts = ([I.Instance(0, 60, 3, p) for p in range(-1, 12)] +      # 13: lanes, d = 2
             [I.Instance(1, 60, 3, p) for p in range(-1, 9)] +       # 10: lanes, d = 3
             [I.Instance(1, 90, 2, p) for p in range(-1, 3)] +       # 4: bundles of 2 + 2
             [I.Instance(0, 100, 4, -1), I.Instance(1, 110, 1, 0)])  # unshared
    ds = te.to_device([s2, s3])
    on, paths, _, _ = _run(te_handle, ds, insts, 4, te.SHARE_LANES)
    assert paths == (23, 4, 2)
    off, _, _, _ = _run(te_handle, ds, insts, 4, te.SHARE_NONE)
    assert torch.equal(off["counts"], on["counts"]) and torch.equal(off["eps"], on["eps"])
    o_te, o_counts, o_eps = oracle.te_batch([s2, s3], insts, 4, want_counts=True)
    np.testing.assert_array_equal(on["eps"].cpu().numpy(), o_eps)
    np.testing.assert_array_equal(on["counts"].cpu().numpy(), o_counts)
    assert np.max(np.abs(on["te"].cpu().numpy() - o_te)) <= TOL


def test_delay_scan_in_lanes_equals_unshared(te_handle):
    """Delays and surrogates of one window share the target part: 5 delays x (1 + 3) = 20
    estimates per window run one per lane."""
    rng = np.random.default_rng(800)
    s = _series(rng, 40, 200, 3, 2, 6, 3)
    ds = te.to_device([s])
    starts = [40, 90]
    te.te_set_sharing(te_handle, te.SHARE_NONE)
    try:
        off = te.te_delay_scan(te_handle, ds[0], starts, 4, 4, 8, 3, 4)
        torch.cuda.synchronize()
    finally:
        te.te_set_sharing(te_handle, te.SHARE_AUTO)
    te.te_set_sharing(te_handle, te.SHARE_LANES)
    try:
        on = te.te_delay_scan(te_handle, ds[0], starts, 4, 4, 8, 3, 4)
        torch.cuda.synchronize()
        assert te.te_last_paths(te_handle)[0] == 2 * 5 * 4
    finally:
        te.te_set_sharing(te_handle, te.SHARE_AUTO)
    assert torch.max(torch.abs(off["te"] - on["te"])).item() <= 1e-9
    assert torch.equal(off["p"], on["p"]) and torch.equal(off["u_best"], on["u_best"])
    for iu, u in enumerate(range(4, 9)):
        su = I.Series(s.src, s.tgt, d=s.d, tau=s.tau, u=u, perms=s.perms)
        o = oracle.te_batch([su], [I.Instance(0, t, 4, -1) for t in starts], 4)
        assert np.max(np.abs(on["te"][iu].cpu().numpy() - o)) <= TOL


def test_bad_permutation_entry_in_lanes_is_flagged(te_handle):
    rng = np.random.default_rng(900)
    s = _series(rng, 30, 40, 2, 1, 2, 9)
    s.perms[4, 11] = s.R + 3
    ds = te.to_device([s])
    te.te_set_sharing(te_handle, te.SHARE_LANES)
    te.te_estimate(te_handle, ds, [I.Instance(0, 10, 3, p) for p in range(-1, 3)] +
                   [I.Instance(0, 10, 3, p) for p in range(5, 9)], 4)
    assert te.te_last_paths(te_handle)[0] == 8
    te.te_sync_status(te_handle)  # entry 4 not used: no flag
    te.te_estimate(te_handle, ds, [I.Instance(0, 10, 3, p) for p in range(-1, 9)], 4)
    assert te.te_last_paths(te_handle)[0] == 10
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_sync_status(te_handle)
    te.te_set_sharing(te_handle, te.SHARE_AUTO)


def test_default_rule_takes_large_groups_of_wide_estimates(te_handle):
    """By default the lane kernel takes groups of 32 or more estimates with d >= 3 only."""
    rng = np.random.default_rng(950)
    s4 = _series(rng, 40, 60, 4, 1, 2, 40)
    s3 = I.Series(s4.src, s4.tgt, d=3, tau=1, u=2, perms=s4.perms)
    # 41 estimates with d = 4 and 41 with d = 3: lanes; the group of 31 (d = 4): bundles; a
    # group of 3 with d = 2: bundles are of one d per batch (the d with most), so it runs unshared
    s2 = I.Series(s4.src, s4.tgt, d=2, tau=1, u=2, perms=s4.perms)
    insts = ([I.Instance(0, 20, 2, p) for p in range(-1, 40)] +
             [I.Instance(0, 30, 2, p) for p in range(-1, 30)] +
             [I.Instance(1, 20, 2, p) for p in range(-1, 40)] +
             [I.Instance(2, 25, 2, p) for p in range(-1, 2)])
    ds = te.to_device([s4, s3, s2])
    on, paths, _, _ = _run(te_handle, ds, insts, 4, te.SHARE_AUTO)
    assert paths == (82, 31, 3)
    o_te, o_counts, o_eps = oracle.te_batch([s4, s3, s2], insts, 4, want_counts=True)
    np.testing.assert_array_equal(on["counts"].cpu().numpy(), o_counts)
    np.testing.assert_array_equal(on["eps"].cpu().numpy(), o_eps)
    assert np.max(np.abs(on["te"].cpu().numpy() - o_te)) <= TOL


def test_lanes_are_deterministic_and_replay(te_handle):
    te.te_set_sharing(te_handle, te.SHARE_LANES)
    w = I.config(3, n_t=2, S=40)
    ds = te.to_device(w.series)
    a = te.te_surrogate_test(te_handle, ds, w.t_starts[0], w.window, w.S, w.k)
    a = {k: v.clone() for k, v in a.items()}
    b = te.te_surrogate_test(te_handle, ds, w.t_starts[0], w.window, w.S, w.k)
    torch.cuda.synchronize()
    assert te.te_last_paths(te_handle)[0] == len(w.instances)
    te.te_set_sharing(te_handle, te.SHARE_AUTO)
    for key in a:
        assert torch.equal(a[key], b[key])


@pytest.mark.parametrize("d,ties,mode", [(3, False, 3), (5, False, 1), (4, True, 3), (2, True, 3)])
def test_strips_equal_unshared_and_oracle(te_handle, d, ties, mode):
    """Groups of 4,500 points (1,500 trials x window 3) are cut into strips of 1,024 by a second
    target coordinate, the last one ragged (404 points): the lane sweeps skip whole strips by the
    second key. Radii and counts equal the unshared search (itself over strips) bit for bit and
    the oracle on sampled estimates; many equal keys included."""
    rng = np.random.default_rng(1000 + 10 * d + int(ties))
    s = _series(rng, 1500, 40, d, 1, 3, 32, ties=ties)
    insts = [I.Instance(0, 12, 3, p) for p in range(-1, 32)]  # 33 estimates
    ds = te.to_device([s])
    off, p0, _, _ = _run(te_handle, ds, insts, 4, te.SHARE_NONE)
    on, p1, ops1, alg1 = _run(te_handle, ds, insts, 4, mode)
    assert p0[0] == 0 and p1[0] == 33 and ops1 < alg1
    assert torch.equal(off["counts"], on["counts"]) and torch.equal(off["eps"], on["eps"])
    assert bool(((off["te"] - on["te"]).abs() <= off["err_bound"] + on["err_bound"]).all())
    N = 4500
    idx = [0, 17, 32]
    o_te, o_counts, o_eps = oracle.te_batch([s], [insts[i] for i in idx], 4, want_counts=True)
    eps = on["eps"].cpu().numpy().reshape(33, N)
    counts = on["counts"].cpu().numpy().reshape(33, 3 * N)
    for j, i in enumerate(idx):
        np.testing.assert_array_equal(eps[i], o_eps[j * N:(j + 1) * N])
        np.testing.assert_array_equal(counts[i], o_counts[3 * j * N:3 * (j + 1) * N])
    assert np.max(np.abs(on["te"].cpu().numpy()[idx] - o_te)) <= TOL


@pytest.mark.parametrize("tau", [2, 3, 4])
def test_every_delay_class(te_handle, tau):
    """tau = 1, 2, 3 are compiled into the lane kernel, any other tau is read at run time: each
    class equals the unshared search and the oracle."""
    rng = np.random.default_rng(1100 + tau)
    s = _series(rng, 45, 80, 3, tau, 3, 11)
    t0 = 3 + 2 * tau + 4
    insts = [I.Instance(0, t0, 3, p) for p in range(-1, 11)]
    _check_against_unshared_and_oracle(te_handle, [s], insts, 4, 12)
