"""Wide embeddings (d = 6..8, joint dimension 13..17) and the Lorenz workloads of Eq. 11 through
the C ABI: radii and counts bit-exact against the CPU oracle (whole point sets where the oracle
finishes in seconds, sampled query points of the paper's 30094-point 17-D chunk), TE within
1e-6 nats, both search modes."""
import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu
TOL = 1e-6


@pytest.mark.parametrize("d", [6, 7, 8])
@pytest.mark.parametrize("k", [4, 8])
@pytest.mark.parametrize("sweep", [True, False])
def test_wide_embedding_matches_oracle(te_handle, d, k, sweep):
    rng = np.random.default_rng(200 + d)
    src, tgt = I.lorenz_pair(rng, 40, 220, coupled=None, burn=300)
    s = I.Series(src, tgt, d=d, tau=2, u=45, perms=I.permutations(rng, 3, 40))
    insts = [I.Instance(0, t, W, p) for t, W in ((100, 5), (150, 3)) for p in (-1, 0, 2)]
    ds = te.to_device([s])
    te.te_set_search(te_handle, sweep)
    try:
        res = te.te_estimate(te_handle, ds, insts, k, want_err=True, want_counts=True)
        torch.cuda.synchronize()
        te.te_sync_status(te_handle)
        swept = te.te_last_work(te_handle)[2]
    finally:
        te.te_set_search(te_handle, True)
    assert swept == sweep
    o_te, o_counts, o_eps = oracle.te_batch([s], insts, k, want_counts=True)
    np.testing.assert_array_equal(res["eps"].cpu().numpy(), o_eps)
    np.testing.assert_array_equal(res["counts"].cpu().numpy(), o_counts)
    assert np.max(np.abs(res["te"].cpu().numpy() - o_te)) <= TOL
    assert np.all(res["err_bound"].cpu().numpy() <= TOL)


def test_mixed_dimensions_above_five_are_refused(te_handle):
    rng = np.random.default_rng(7)
    src, tgt = I.lorenz_pair(rng, 20, 200, coupled=None, burn=200)
    ds = te.to_device([I.Series(src, tgt, d=6, tau=1, u=45), I.Series(src, tgt, d=2, tau=1, u=45)])
    with pytest.raises(te.TEError, match="TE_ENOTIMPL"):
        te.te_estimate(te_handle, ds, [I.Instance(0, 100, 5, -1), I.Instance(1, 100, 5, -1)], 4)


def test_paper_chunk_sampled_points(te_handle):
    """Two chunks of 30094 points x 17-D (d = 8), the launch the benchmark times: radii and
    counts of 96 seeded query points per chunk against the oracle's per-point evaluation."""
    w = I.paper_chunk(chunks=2)
    ds = te.to_device(w.series)
    res = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=True)
    torch.cuda.synchronize()
    te.te_sync_status(te_handle)
    N = w.n_points(w.instances[0])
    eps = res["eps"].cpu().numpy().reshape(2, N)
    counts = res["counts"].cpu().numpy().reshape(2, 3, N)
    s = w.series[0]
    rng = np.random.default_rng(31)
    for c, it in enumerate(w.instances):
        perm = None if it.perm < 0 else s.perms[it.perm]
        pts = oracle.embed(s.src, s.tgt, s.d, s.tau, s.u, it.t_start, it.window, perm)
        idx = np.sort(rng.choice(N, 96, replace=False))
        e, cnt = oracle.points_at(pts, s.d, s.d, w.k, idx)
        np.testing.assert_array_equal(eps[c, idx], e)
        np.testing.assert_array_equal(counts[c][:, idx], cnt)
    assert np.all(res["err_bound"].cpu().numpy() <= TOL)


def test_nonstationary_lorenz_delay_scan(te_handle):
    """Fig. 6: coupling only during samples 1000..2000; windows 200..450, 1600..1850, 2750..3000,
    delays 35..55. In the coupled window the TE at the reconstructed delay is significant and the
    delay is within 10 % of the true 45 samples (the paper: 49); in the others no scanned delay is
    significant. Radii and counts of the coupled window's original estimate at u = 45 are checked
    on sampled query points against the oracle."""
    w = I.lorenz_analysis(S=50)
    ds = te.to_device(w.series)
    r = te.te_delay_scan(te_handle, ds[0], w.t_starts[0], w.window, 35, 55, w.S, w.k)
    torch.cuda.synchronize()
    ub = r["u_best"].cpu().numpy()
    p = r["p"].cpu().numpy()
    assert p[ub[1] - 35, 1] == 0.0 and abs(int(ub[1]) - 45) <= 4
    assert p[:, 0].min() >= 0.05 and p[:, 2].min() >= 0.05
    s = w.series[0]
    su = I.Series(s.src, s.tgt, d=s.d, tau=s.tau, u=45, perms=s.perms)
    res = te.te_estimate(te_handle, te.to_device([su]), [I.Instance(0, 1600, 250, -1)], w.k, want_counts=True)
    torch.cuda.synchronize()
    assert abs(res["te"][0].item() - r["te"][45 - 35, 1].item()) <= 1e-12
    pts = oracle.embed(s.src, s.tgt, s.d, s.tau, 45, 1600, 250)
    idx = np.sort(np.random.default_rng(4).choice(pts.shape[0], 64, replace=False))
    e, cnt = oracle.points_at(pts, s.d, s.d, w.k, idx)
    np.testing.assert_array_equal(res["eps"].cpu().numpy()[idx], e)
    np.testing.assert_array_equal(res["counts"].cpu().numpy().reshape(3, -1)[:, idx], cnt)


def test_lorenz_robustness_delay_scan(te_handle):
    """Fig. 8: constant coupling, delays 30..60, point sets of 600 .. 30000 points (whole
    repetitions). With 2000 points or more the TE at the reconstructed delay is significant, and
    with 30000 points the delay is within 3 samples of 45. The TE of the 2000-point set at u = 45
    matches the oracle."""
    rob = I.lorenz_robustness(S=20)
    ub = {}
    for M, w in rob.items():
        ds = te.to_device(w.series)
        r = te.te_delay_scan(te_handle, ds[0], w.t_starts[0], w.window, 30, 60, w.S, w.k)
        torch.cuda.synchronize()
        ub[M] = int(r["u_best"][0])
        if M >= 2000:
            assert r["p"][ub[M] - 30, 0].item() == 0.0
        if M == 2000:
            s = w.series[0]
            su = I.Series(s.src, s.tgt, d=s.d, tau=s.tau, u=45, perms=s.perms)
            o = oracle.te_batch([su], [I.Instance(0, 100, 200, -1)], w.k)
            assert abs(r["te"][45 - 30, 0].item() - o[0]) <= TOL
    assert abs(ub[30000] - 45) <= 3, ub


@pytest.mark.parametrize("N,W,ties", [(8193, 3, False), (20000, 4, True), (40961, 13, False), (65536, 16, False)])
def test_sweep_above_one_sort_run_equals_exhaustive(te_handle, N, W, ties):
    """Point counts past one shared-memory sort run (8192): the sort merges runs through global
    memory (1 to 3 passes, ragged last runs, many equal keys); the sweep built on that order must
    give exactly the exhaustive search's radii and counts."""
    rng = np.random.default_rng(N)
    R = N // W
    if ties:
        src = rng.integers(0, 6, (R, 40)).astype(np.float32)
        tgt = rng.integers(0, 6, (R, 40)).astype(np.float32)
    else:
        src = rng.standard_normal((R, 40)).astype(np.float32)
        tgt = rng.standard_normal((R, 40)).astype(np.float32)
    s = I.Series(src, tgt, d=2, tau=1, u=3, perms=I.permutations(rng, 1, R))
    insts = [I.Instance(0, 10, W, -1), I.Instance(0, 10, W, 0)]
    ds = te.to_device([s])
    te.te_set_search(te_handle, False)
    try:
        ref = te.te_estimate(te_handle, ds, insts, 4, want_counts=True)
    finally:
        te.te_set_search(te_handle, True)
    got = te.te_estimate(te_handle, ds, insts, 4, want_counts=True)
    torch.cuda.synchronize()
    pairs, _, swept = te.te_last_work(te_handle)
    assert swept and 0 < pairs
    assert torch.equal(ref["eps"], got["eps"]) and torch.equal(ref["counts"], got["counts"])
    assert torch.max(torch.abs(ref["te"] - got["te"])).item() <= 1e-9


def test_paper_chunk_sweep_equals_exhaustive(te_handle):
    w = I.paper_chunk(chunks=2)
    ds = te.to_device(w.series)
    te.te_set_search(te_handle, False)
    try:
        ref = te.te_estimate(te_handle, ds, w.instances, w.k, want_counts=True)
    finally:
        te.te_set_search(te_handle, True)
    got = te.te_estimate(te_handle, ds, w.instances, w.k, want_counts=True)
    torch.cuda.synchronize()
    assert te.te_last_work(te_handle)[2]
    assert torch.equal(ref["eps"], got["eps"]) and torch.equal(ref["counts"], got["counts"])


@pytest.mark.parametrize("shape", [(256, 1), (512, 1)])
def test_paper_chunk_strips_equal_exhaustive(te_handle, shape):
    """With a CTA block that divides a strip, the unshared tiled sweep of the 17-D chunk runs over
    strips (second key y_{t'-1-tau}); radii and counts equal the exhaustive search."""
    w = I.paper_chunk(chunks=2)
    ds = te.to_device(w.series)
    te.te_set_search(te_handle, False)
    try:
        ref = te.te_estimate(te_handle, ds, w.instances, w.k, want_counts=True)
    finally:
        te.te_set_search(te_handle, True)
    te.te_set_launch_config(te_handle, *shape)
    try:
        got = te.te_estimate(te_handle, ds, w.instances, w.k, want_counts=True)
        torch.cuda.synchronize()
        pairs, _, swept = te.te_last_work(te_handle)
    finally:
        te.te_set_launch_config(te_handle, 0, 0)
    N = w.n_points(w.instances[0])
    assert swept and pairs < 0.25 * 2 * 2 * N * N
    assert torch.equal(ref["eps"], got["eps"]) and torch.equal(ref["counts"], got["counts"])


@pytest.mark.parametrize("N,W,ties", [(20000, 4, True), (40961, 13, False)])
def test_tiled_strips_equal_exhaustive(te_handle, N, W, ties):
    """Unshared estimates too large to stage whole (d = 2), CTA blocks of 256 queries: the tiled
    sweep over strips equals the exhaustive search, many equal keys included."""
    rng = np.random.default_rng(N + 5)
    R = N // W
    if ties:
        src = rng.integers(0, 6, (R, 40)).astype(np.float32)
        tgt = rng.integers(0, 6, (R, 40)).astype(np.float32)
    else:
        src = rng.standard_normal((R, 40)).astype(np.float32)
        tgt = rng.standard_normal((R, 40)).astype(np.float32)
    s = I.Series(src, tgt, d=2, tau=1, u=3, perms=I.permutations(rng, 1, R))
    insts = [I.Instance(0, 10, W, -1), I.Instance(0, 10, W, 0)]
    ds = te.to_device([s])
    te.te_set_sharing(te_handle, False)
    try:
        te.te_set_search(te_handle, False)
        try:
            ref = te.te_estimate(te_handle, ds, insts, 4, want_counts=True)
        finally:
            te.te_set_search(te_handle, True)
        te.te_set_launch_config(te_handle, 128, 2)
        got = te.te_estimate(te_handle, ds, insts, 4, want_counts=True)
        torch.cuda.synchronize()
    finally:
        te.te_set_launch_config(te_handle, 0, 0)
        te.te_set_sharing(te_handle, True)
    assert torch.equal(ref["eps"], got["eps"]) and torch.equal(ref["counts"], got["counts"])
    assert torch.max(torch.abs(ref["te"] - got["te"])).item() <= 1e-9
