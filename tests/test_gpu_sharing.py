"""Target-part sharing (the bundle kernel): estimates that share y_t and y- (the original and its
trial-shuffled surrogates, every scanned delay u) run in bundles that compute the target part of
each distance and count once. Per-point radii and counts must equal the unshared search and the
CPU oracle bit for bit, TE within 1e-6 nats of the oracle; bundles of every size 2..3, ragged
point counts, mixed embedding dimensions, the delay scan and a bad permutation entry.
Bundles hold up to 3 estimates (never 1: a remainder of one turns the last two bundles into 2 + 2).
Groups of 8 or more estimates with d >= 2 go to the lane kernel by default (tests/test_gpu_lanes.py);
the tests here ask for bundles only (te.SHARE_BUNDLES) where their groups are that large."""
import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _estimate(h, ds, insts, k, sharing):
    te.te_set_sharing(h, te.SHARE_BUNDLES if sharing is True else sharing)
    try:
        res = te.te_estimate(h, ds, insts, k, want_err=True, want_counts=True)
        torch.cuda.synchronize()
        te.te_sync_status(h)
        ops, bundles = te.te_last_alu_ops(h)
        pairs, alg_ops, swept = te.te_last_work(h)
    finally:
        te.te_set_sharing(h, True)
    return res, bundles, ops, alg_ops, swept


def _oracle_check(series, insts, k, res):
    o_te, o_counts, o_eps = oracle.te_batch(series, insts, k, want_counts=True)
    np.testing.assert_array_equal(res["eps"].cpu().numpy(), o_eps)
    np.testing.assert_array_equal(res["counts"].cpu().numpy(), o_counts)
    assert np.max(np.abs(res["te"].cpu().numpy() - o_te)) <= TOL
    assert np.all(res["err_bound"].cpu().numpy() <= TOL)


def test_shared_equals_unshared_and_oracle(te_handle):
    w = I.config(3, n_t=2, S=9)  # 10 estimates per start: bundles of 3, 3, 2, 2
    ds = te.to_device(w.series)
    off, b0, ops0, alg0, _ = _estimate(te_handle, ds, w.instances, w.k, False)
    on, b1, ops1, alg1, swept = _estimate(te_handle, ds, w.instances, w.k, True)
    assert swept and b0 == 0 and b1 == 8
    assert ops0 == alg0 and ops1 < alg1
    assert torch.equal(off["counts"], on["counts"]) and torch.equal(off["eps"], on["eps"])
    assert torch.max(torch.abs(off["te"] - on["te"])).item() <= 1e-12
    idx = [0, 1, 4, 9, 10, 15, 19]
    sub = [w.instances[i] for i in idx]
    res = te.te_estimate(te_handle, ds, sub, w.k, want_err=True, want_counts=True)
    torch.cuda.synchronize()
    assert te.te_last_alu_ops(te_handle)[1] == 3  # starts 0 and 1: {0,1}, {4,9}, {10,15,19}
    _oracle_check(w.series, sub, w.k, res)


@pytest.mark.parametrize("R,window", [(37, 3), (64, 2), (11, 1)])
def test_every_bundle_size_and_ragged_point_counts(te_handle, R, window):
    rng = np.random.default_rng(100 + R)
    src, tgt = I.ar2_pair(rng, R, 120)
    s = I.Series(src, tgt, d=3, tau=1, u=5, perms=I.permutations(rng, 9, R))
    # starts with 2, 3, 5, 6 and 9 estimates: bundles 2 | 3 | 3+2 | 3+3 | 3+3+3
    sizes = {20: 2, 30: 3, 40: 5, 50: 6, 60: 9}
    insts = [I.Instance(0, t, window, p) for t, n in sizes.items() for p in range(-1, n - 1)]
    ds = te.to_device([s])
    res, bundles, _, _, _ = _estimate(te_handle, ds, insts, 4, True)
    assert bundles == 1 + 1 + 2 + 2 + 3
    _oracle_check([s], insts, 4, res)


def test_mixed_dimensions_share_one_dimension(te_handle):
    rng = np.random.default_rng(5)
    src, tgt = I.ar2_pair(rng, 50, 150)
    perms = I.permutations(rng, 4, 50)
    s2 = I.Series(src, tgt, d=2, tau=1, u=5, perms=perms)
    s3 = I.Series(src, tgt, d=3, tau=2, u=5, perms=perms)
    insts = ([I.Instance(0, 60, 3, p) for p in range(-1, 4)] + [I.Instance(1, 60, 3, p) for p in range(-1, 4)] +
             [I.Instance(1, 90, 2, p) for p in range(-1, 2)] + [I.Instance(0, 100, 4, -1)])
    ds = te.to_device([s2, s3])
    res, bundles, _, _, _ = _estimate(te_handle, ds, insts, 4, True)
    assert bundles == 3  # d = 3 (8 estimates: 3+2 and 3); d = 2 and the single estimate unshared
    _oracle_check([s2, s3], insts, 4, res)


def test_delay_scan_shares_the_target_part_across_delays(te_handle):
    w = I.ar1_analysis("unidirectional", S=6, R=24, window=40, n_windows=2)
    ds = te.to_device(w.series)
    starts = w.t_starts[0]
    te.te_set_sharing(te_handle, False)
    try:
        off = te.te_delay_scan(te_handle, ds[0], starts, w.window, 8, 12, w.S, w.k)
        torch.cuda.synchronize()
    finally:
        te.te_set_sharing(te_handle, True)
    on = te.te_delay_scan(te_handle, ds[0], starts, w.window, 8, 12, w.S, w.k)
    torch.cuda.synchronize()
    assert te.te_last_alu_ops(te_handle)[1] > 0
    assert torch.max(torch.abs(off["te"] - on["te"])).item() <= 1e-12
    assert torch.equal(off["p"], on["p"]) and torch.equal(off["u_best"], on["u_best"])
    s = w.series[0]
    for iu, u in enumerate(range(8, 13)):
        su = I.Series(s.src, s.tgt, d=s.d, tau=s.tau, u=u, perms=s.perms)
        o = oracle.te_batch([su], [I.Instance(0, t, w.window, -1) for t in starts], w.k)
        assert np.max(np.abs(on["te"][iu].cpu().numpy() - o)) <= TOL


def test_bad_permutation_entry_in_a_bundle_is_flagged(te_handle):
    w = I.config(1)
    s = w.series[0]
    bad = I.permutations(np.random.default_rng(1), 3, s.R)
    bad[2, 7] = s.R + 5
    s.perms = bad
    ds = te.to_device([s])
    te.te_estimate(te_handle, ds, [I.Instance(0, 100, 5, p) for p in (-1, 0, 1)], 4)
    assert te.te_last_alu_ops(te_handle)[1] == 1
    te.te_sync_status(te_handle)
    te.te_estimate(te_handle, ds, [I.Instance(0, 100, 5, p) for p in (0, 2)], 4)
    assert te.te_last_alu_ops(te_handle)[1] == 1
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_sync_status(te_handle)


def test_tiled_bundles_match_unshared_and_oracle(te_handle):
    """Estimates too large for shared memory on their own (7500 points x 7 = 210 KB; a bundle of
    three 390 KB) run in tiled bundles; radii and counts equal the unshared search bit for bit and
    the oracle on sampled estimates."""
    w = I.config(3, n_t=2, S=4, R=2500)  # 5 estimates per start: bundles of 3 + 2
    ds = te.to_device(w.series)
    off, b0, _, _, _ = _estimate(te_handle, ds, w.instances, w.k, False)
    on, b1, ops1, alg1, swept = _estimate(te_handle, ds, w.instances, w.k, True)
    assert swept and b0 == 0 and b1 == 4 and ops1 < alg1
    assert torch.equal(off["counts"], on["counts"]) and torch.equal(off["eps"], on["eps"])
    assert torch.max(torch.abs(off["te"] - on["te"])).item() <= 1e-12
    idx = [0, 3, 7]
    o_te, o_counts, o_eps = oracle.te_batch(w.series, [w.instances[i] for i in idx], w.k, want_counts=True)
    N = w.n_points(w.instances[0])
    eps = on["eps"].cpu().numpy().reshape(-1, N)
    counts = on["counts"].cpu().numpy().reshape(-1, 3 * N)
    for j, i in enumerate(idx):
        np.testing.assert_array_equal(eps[i], o_eps[j * N:(j + 1) * N])
        np.testing.assert_array_equal(counts[i], o_counts[3 * j * N:3 * (j + 1) * N])
    assert np.max(np.abs(on["te"].cpu().numpy()[idx] - o_te)) <= TOL


def test_delay_scan_with_tiled_bundles(te_handle):
    """A delay scan whose windows are too large to stay resident (Lorenz, 150 repetitions x 250
    samples = 37,500 points, d = 4) shares the target part across delays and surrogates in tiled
    bundles; the scan equals the unshared one, and the original at u = 45 matches the oracle on
    sampled query points. AR(1) windows (15,000 points, d = 1) stay resident and unshared."""
    w = I.lorenz_analysis(S=2)
    ds = te.to_device(w.series)
    starts = w.t_starts[0][1:2]
    te.te_set_sharing(te_handle, False)
    try:
        off = te.te_delay_scan(te_handle, ds[0], starts, w.window, 44, 46, w.S, w.k)
        torch.cuda.synchronize()
        te.te_set_sharing(te_handle, te.SHARE_BUNDLES)
        on = te.te_delay_scan(te_handle, ds[0], starts, w.window, 44, 46, w.S, w.k)
        torch.cuda.synchronize()
        assert te.te_last_alu_ops(te_handle)[1] == 3  # 3 delays x 3 estimates = 9
    finally:
        te.te_set_sharing(te_handle, True)
    assert torch.max(torch.abs(off["te"] - on["te"])).item() <= 1e-12
    assert torch.equal(off["p"], on["p"]) and torch.equal(off["u_best"], on["u_best"])
    wa = I.ar1_analysis("unidirectional", S=4, R=50, window=300, n_windows=1)
    dsa = te.to_device(wa.series)
    te.te_delay_scan(te_handle, dsa[0], wa.t_starts[0], wa.window, 8, 10, wa.S, wa.k)
    torch.cuda.synchronize()
    assert te.te_last_alu_ops(te_handle)[1] == 0


@pytest.mark.parametrize("d,ties", [(1, False), (1, True), (2, True)])
def test_tiled_bundles_with_strips_equal_unshared(te_handle, d, ties):
    """Tiled bundles over sort groups cut into strips (second key y_t for d = 1, which prunes only
    the kNN pass; y_{t'-1-tau} for d >= 2, which prunes both passes): radii and counts equal the
    unshared search, many equal keys included."""
    rng = np.random.default_rng(77 + d + (10 if ties else 0))
    R, W = 5000, 4  # 20,000 points: too large to stage whole even alone
    if ties:
        src = rng.integers(0, 6, (R, 40)).astype(np.float32)
        tgt = rng.integers(0, 6, (R, 40)).astype(np.float32)
    else:
        src, tgt = I.ar2_pair(rng, R, 40)
    s = I.Series(src, tgt, d=d, tau=2, u=3, perms=I.permutations(rng, 4, R))
    insts = [I.Instance(0, 15, W, p) for p in (-1, 0, 1, 2, 3)]
    ds = te.to_device([s])
    off, b0, _, _, _ = _estimate(te_handle, ds, insts, 4, False)
    on, b1, _, _, _ = _estimate(te_handle, ds, insts, 4, True)
    assert b0 == 0 and b1 == 2
    assert torch.equal(off["counts"], on["counts"]) and torch.equal(off["eps"], on["eps"])
    assert torch.max(torch.abs(off["te"] - on["te"])).item() <= 1e-12


@pytest.mark.parametrize("ties", [False, True])
def test_resident_bundles_with_strips_equal_unshared(te_handle, ties):
    """Resident bundles over a sort group of 6,000 points (d = 1: 5 columns x 6,000 = 120 KB per
    bundle) cut into strips: radii and counts equal the unshared search (itself over strips)."""
    rng = np.random.default_rng(91 + (1 if ties else 0))
    R, W = 2000, 3
    if ties:
        src = rng.integers(0, 6, (R, 40)).astype(np.float32)
        tgt = rng.integers(0, 6, (R, 40)).astype(np.float32)
    else:
        src, tgt = I.ar2_pair(rng, R, 40)
    s = I.Series(src, tgt, d=1, tau=1, u=2, perms=I.permutations(rng, 4, R))
    insts = [I.Instance(0, 12, W, p) for p in (-1, 0, 1, 2, 3)]
    ds = te.to_device([s])
    off, b0, _, _, _ = _estimate(te_handle, ds, insts, 4, False)
    on, b1, _, _, _ = _estimate(te_handle, ds, insts, 4, True)
    assert b0 == 0 and b1 == 2
    assert torch.equal(off["counts"], on["counts"]) and torch.equal(off["eps"], on["eps"])
    assert torch.max(torch.abs(off["te"] - on["te"])).item() <= 1e-12
