"""Parity of the batched persistent path (te_estimate, te_surrogate_test) with the CPU oracle
through the C ABI: per-point kNN radii and the three neighbour counts bit-exact, TE within
1e-6 nats, p-values equal.

The tolerance 1e-6 nats is the target the method's precision reading sets; the device sums
digamma terms in compensated FP32 with an FP64 final mean, and the reported error bound must
itself stay below it.  Workloads: every configuration at its full point count N and joint
dimension D, in the launch configuration the benchmark uses, on seeded instance samples
(full batches are launched on the GPU, the oracle recomputes sampled instances)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _check_against_oracle(w, res, idx, check_counts=True):
    """Compare sampled instances idx of a te_estimate result with the oracle."""
    insts = [w.instances[i] for i in idx]
    o_te, o_counts, o_eps = oracle.te_batch(w.series, insts, w.k, want_counts=True)
    g_te = res["te"].cpu().numpy()
    err = res["err_bound"].cpu().numpy()
    # per-instance point offsets in the concatenated outputs
    off = np.zeros(len(w.instances) + 1, dtype=np.int64)
    for i, it in enumerate(w.instances):
        off[i + 1] = off[i] + w.n_points(it)
    if check_counts:
        g_counts = res["counts"].cpu().numpy()
        g_eps = res["eps"].cpu().numpy()
        po = 0
        for j, i in enumerate(idx):
            n = w.n_points(w.instances[i])
            np.testing.assert_array_equal(g_eps[off[i]:off[i] + n], o_eps[po:po + n])
            np.testing.assert_array_equal(g_counts[3 * off[i]:3 * off[i] + 3 * n],
                                          o_counts[3 * po:3 * po + 3 * n])
            po += n
    d = np.abs(g_te[idx] - o_te)
    assert d.max() <= TOL, d.max()
    assert np.all(err[idx] <= TOL)
    return d.max()


def _run(te_handle, w, want_counts=True):
    ds = te.to_device(w.series)
    res = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=want_counts)
    torch.cuda.synchronize()
    te.te_sync_status(te_handle)
    return ds, res


def test_c1_full(te_handle):
    w = I.config(1)
    _, res = _run(te_handle, w)
    _check_against_oracle(w, res, [0])


def test_c2_full_all_time_points(te_handle):
    w = I.config(2)
    _, res = _run(te_handle, w)
    _check_against_oracle(w, res, list(range(len(w.instances))))


def test_c3_full_batch_sampled(te_handle):
    w = I.config(3)
    _, res = _run(te_handle, w)
    idx = I.sample_instances(w, 24, seed=3)
    idx = sorted(set(idx) | {0, 1, 1000, len(w.instances) - 1})
    _check_against_oracle(w, res, idx)


def test_c4_full_uneven_batch_sampled(te_handle):
    w = I.config(4)
    _, res = _run(te_handle, w)
    _check_against_oracle(w, res, I.sample_instances(w, 12, seed=4))


def test_c5_full_size_instances_sampled(te_handle):
    # full N = 12000 x 11-D instances, two time points x (1 + 200 surrogates) launched
    w = I.config(5, n_t=2)
    _, res = _run(te_handle, w)
    _check_against_oracle(w, res, [0, 7, 201 + 150])


def test_surrogate_test_matches_oracle(te_handle):
    w = I.config(3, n_t=3, S=40)
    ds = te.to_device(w.series)
    out = te.te_surrogate_test(te_handle, ds, w.t_starts[0], w.window, w.S, w.k)
    torch.cuda.synchronize()
    o_te = oracle.te_batch(w.series, w.instances, w.k)
    S = w.S
    for j in range(len(w.t_starts[0])):
        blk = o_te[j * (S + 1):(j + 1) * (S + 1)]
        assert abs(out["te_orig"][0, j].item() - blk[0]) <= TOL
        assert np.max(np.abs(out["te_surr"][0, j].cpu().numpy() - blk[1:])) <= TOL
        # the p-value is decided in FP64 on both sides; no surrogate lies within TOL of TE_0
        assert np.min(np.abs(blk[1:] - blk[0])) > 2 * TOL
        assert out["p"][0, j].item() == oracle.pvalue(blk[0], blk[1:])


def test_surrogate_test_two_series_and_zero_surrogates(te_handle):
    a = I.config(1)
    rng = np.random.default_rng(9)
    src, tgt = I.ar2_pair(rng, 90, 300, coupling_start=None)
    s2 = I.Series(src, tgt, d=2, tau=1, u=5, perms=I.permutations(rng, 5, 90))
    s1 = a.series[0]
    s1.perms = I.permutations(rng, 5, s1.R)
    ds = te.to_device([s1, s2])
    out = te.te_surrogate_test(te_handle, ds, [50, 120], 5, 5, 4)
    out0 = te.te_surrogate_test(te_handle, ds, [50, 120], 5, 0, 4)
    torch.cuda.synchronize()
    insts = [I.Instance(si, t, 5, p) for si in (0, 1) for t in (50, 120) for p in [-1, 0, 1, 2, 3, 4]]
    o = oracle.te_batch([s1, s2], insts, 4).reshape(2, 2, 6)
    np.testing.assert_allclose(out["te_orig"].cpu().numpy(), o[:, :, 0], atol=TOL, rtol=0)
    np.testing.assert_allclose(out["te_surr"].cpu().numpy(), o[:, :, 1:], atol=TOL, rtol=0)
    np.testing.assert_allclose(out0["te_orig"].cpu().numpy(), o[:, :, 0], atol=TOL, rtol=0)
    assert torch.isnan(out0["p"]).all()


@pytest.mark.parametrize("threads,qpt", [(64, 2), (96, 4), (160, 4), (256, 2), (512, 4), (1024, 2), (640, 1), (0, 0)])
def test_launch_shape_does_not_change_counts(te_handle, threads, qpt):
    w = I.config(4, n_pairs=6, n_t=3)
    ds = te.to_device(w.series)
    te.te_set_launch_config(te_handle, 0, 0)
    ref = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=True)
    te.te_set_launch_config(te_handle, threads, qpt)
    try:
        got = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=True)
    finally:
        te.te_set_launch_config(te_handle, 0, 0)
    torch.cuda.synchronize()
    assert torch.equal(ref["counts"], got["counts"])
    assert torch.equal(ref["eps"], got["eps"])
    assert torch.max(torch.abs(ref["te"] - got["te"])).item() <= 1e-9


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 16])
def test_other_k(te_handle, k):
    w = I.config(3, n_t=1, S=5, R=120)
    w.k = k
    _, res = _run(te_handle, w)
    _check_against_oracle(w, res, list(range(len(w.instances))))


def test_degenerate_minimum_points_and_ties(te_handle):
    # N = k + 1 points; integer-valued series (many exact distance ties and eps = 0 cases)
    rng = np.random.default_rng(12)
    src = rng.integers(0, 3, size=(5, 40)).astype(np.float32)
    tgt = rng.integers(0, 3, size=(5, 40)).astype(np.float32)
    s = I.Series(src, tgt, d=1, tau=1, u=1, perms=I.permutations(rng, 3, 5))
    w = I.Workload("tiny", [s], [I.Instance(0, t, 1, p) for t in (3, 10, 30) for p in (-1, 0, 1, 2)], k=4)
    _, res = _run(te_handle, w)
    _check_against_oracle(w, res, list(range(len(w.instances))))
    w2 = I.Workload("ties", [s], [I.Instance(0, t, W, -1) for t in (5, 20) for W in (2, 5, 9)], k=2)
    _, res2 = _run(te_handle, w2)
    _check_against_oracle(w2, res2, list(range(len(w2.instances))))


def test_deterministic_and_graph_replay(te_handle):
    w = I.config(3, n_t=2, S=30)
    ds = te.to_device(w.series)
    out = torch.empty(len(w.instances), dtype=torch.float64, device="cuda")
    a = te.te_estimate(te_handle, ds, w.instances, w.k, te=out).clone()
    n1 = te.te_last_launch_count(te_handle)
    b = te.te_estimate(te_handle, ds, w.instances, w.k, te=out).clone()  # graph replay
    c = te.te_estimate(te_handle, ds, w.instances, w.k)                  # new output: re-capture
    torch.cuda.synchronize()
    swept = te.te_last_work(te_handle)[2]
    lanes = te.te_last_paths(te_handle)[0] > 0
    # persistent kernel + finalisation (+ the sweep's sort pre-pass, + the lane kernel's pre-pass)
    assert n1 == 2 + int(swept) + int(lanes)
    assert torch.equal(a, b) and torch.equal(a, c)


def test_profiling_hook_and_launch_count(te_handle):
    w = I.config(3, n_t=1, S=100)
    ds = te.to_device(w.series)
    te.te_set_profiling(te_handle, True)
    try:
        te.te_surrogate_test(te_handle, ds, w.t_starts[0], w.window, w.S, w.k)
        ms = te.te_last_kernel_ms(te_handle)
        assert ms > 0
        swept = te.te_last_work(te_handle)[2]
        lanes = te.te_last_paths(te_handle)[0] > 0
        assert te.te_last_launch_count(te_handle) == 3 + int(swept) + int(lanes)
    finally:
        te.te_set_profiling(te_handle, False)


def test_bad_permutation_entry_is_flagged_not_read(te_handle):
    w = I.config(1)
    s = w.series[0]
    bad = I.permutations(np.random.default_rng(1), 2, s.R)
    bad[1, 7] = s.R + 5
    s.perms = bad
    ds = te.to_device([s])
    te.te_estimate(te_handle, ds, [I.Instance(0, 100, 5, 0)], 4)
    te.te_sync_status(te_handle)
    te.te_estimate(te_handle, ds, [I.Instance(0, 100, 5, 1)], 4)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_sync_status(te_handle)


def test_argument_errors_launch_nothing(te_handle):
    w = I.config(1)
    ds = te.to_device(w.series)
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    cases = [
        ([I.Instance(0, 2, 5, -1)], 4, "TE_ERANGE"),     # target past before sample 0
        ([I.Instance(0, 298, 5, -1)], 4, "TE_ERANGE"),   # window past the last sample
        ([I.Instance(1, 100, 5, -1)], 4, "TE_EINVAL"),   # no such series
        ([I.Instance(0, 100, 5, 3)], 4, "TE_EINVAL"),    # no such surrogate
        ([I.Instance(0, 100, 5, -1)], 0, "TE_EINVAL"),   # k < 1
        ([I.Instance(0, 100, 5, -1)], 17, "TE_EINVAL"),  # k > 16
    ]
    for insts, k, code in cases:
        with pytest.raises(te.TEError, match=code):
            te.te_estimate(te_handle, ds, insts, k, te=out)
    big = I.Series(np.zeros((20000, 20), np.float32), np.zeros((20000, 20), np.float32), d=1, tau=1, u=1)
    with pytest.raises(te.TEError, match="TE_ENOTIMPL"):
        te.te_estimate(te_handle, te.to_device([big]), [I.Instance(0, 5, 4, -1)], 4)
    torch.cuda.synchronize()
    assert out.item() == 7.0


def test_caller_outputs_are_checked_before_any_launch(te_handle):
    w = I.config(3, n_t=2, S=3)
    ds = te.to_device(w.series)
    n = len(w.instances)
    for bad, err in ((torch.zeros(n - 1, dtype=torch.float64, device="cuda"), ValueError),
                     (torch.zeros(n, dtype=torch.float32, device="cuda"), TypeError),
                     (torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2], ValueError),
                     (torch.zeros(n, dtype=torch.float64), TypeError)):
        with pytest.raises(err):
            te.te_estimate(te_handle, ds, w.instances, w.k, te=bad)
    out = {"te_orig": torch.zeros((1, 2), dtype=torch.float64, device="cuda"),
           "te_surr": torch.zeros((1, 2, 2), dtype=torch.float64, device="cuda"),  # S = 3 needed
           "p": torch.zeros((1, 2), dtype=torch.float64, device="cuda")}
    with pytest.raises(ValueError, match="te_surr"):
        te.te_surrogate_test(te_handle, ds, w.t_starts[0], w.window, w.S, w.k, out=out)
    torch.cuda.synchronize()
    assert float(out["te_surr"].abs().sum()) == 0.0


def test_per_instance_launch_mode_is_bit_identical(te_handle):
    w = I.config(4, n_pairs=5, n_t=2)
    ds = te.to_device(w.series)
    ref = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=True)
    te.te_set_batching(te_handle, True)
    try:
        got = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=True)
        n = te.te_last_launch_count(te_handle)
    finally:
        te.te_set_batching(te_handle, False)
    torch.cuda.synchronize()
    swept = te.te_last_work(te_handle)[2]
    assert n == len(w.instances) + 1 + int(swept)
    assert torch.equal(ref["counts"], got["counts"]) and torch.equal(ref["eps"], got["eps"])
    assert torch.equal(ref["te"], got["te"])


def test_per_instance_launch_mode_with_resident_and_shared_estimates(te_handle):
    # C3 shapes: in one launch the estimates share their target part (bundles); per instance
    # they run unshared, so the partial sums are grouped differently: counts and eps stay
    # bit-identical, TE agrees within the error bound
    w = I.config(3, n_t=2, S=20)
    ds = te.to_device(w.series)
    ref = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=True)
    paths = te.te_last_paths(te_handle)
    assert paths[0] + paths[1] == len(w.instances)
    te.te_set_batching(te_handle, True)
    try:
        got = te.te_estimate(te_handle, ds, w.instances, w.k, want_err=True, want_counts=True)
    finally:
        te.te_set_batching(te_handle, False)
    torch.cuda.synchronize()
    assert torch.equal(ref["counts"], got["counts"]) and torch.equal(ref["eps"], got["eps"])
    diff = (ref["te"] - got["te"]).abs()
    assert bool((diff <= ref["err_bound"] + got["err_bound"]).all())


def test_autotune_picks_a_shape_caches_it_and_keeps_results(te_handle, tmp_path):
    w = I.config(3, n_t=2, S=60)
    ds = te.to_device(w.series)
    ref = te.te_estimate(te_handle, ds, w.instances, w.k, want_counts=True)
    cache = str(tmp_path / "tune.json")
    h2 = te.Handle(0)
    try:
        t, q = te.te_autotune(h2, ds, w.instances, w.k, cache_path=cache)
        assert t % 32 == 0 and 64 <= t <= 512 and q in (2, 4)
        got = te.te_estimate(h2, ds, w.instances, w.k, want_counts=True)
        torch.cuda.synchronize()
        assert torch.equal(ref["counts"], got["counts"]) and torch.equal(ref["eps"], got["eps"])
        assert torch.max(torch.abs(ref["te"] - got["te"])).item() <= 1e-9
        import json
        entries = json.load(open(cache))
        assert any(v["threads"] == t and v["qpt"] == q for v in entries.values())
    finally:
        h2.close()
    h3 = te.Handle(0)  # a fresh handle reads the cache instead of timing again
    try:
        assert te.te_autotune(h3, ds, w.instances, w.k, cache_path=cache) == (t, q)
    finally:
        h3.close()


@pytest.mark.parametrize("case", ["c3", "c4", "ties", "k1", "k16", "ar1", "c5"])
def test_sorted_sweep_equals_exhaustive_search(te_handle, case):
    if case == "c3":
        w = I.config(3, n_t=2, S=30)
    elif case == "c4":
        w = I.config(4, n_pairs=6, n_t=3)
    elif case == "ties":
        rng = np.random.default_rng(31)
        src = rng.integers(0, 4, size=(60, 50)).astype(np.float32)
        tgt = rng.integers(0, 4, size=(60, 50)).astype(np.float32)
        s = I.Series(src, tgt, d=2, tau=1, u=2, perms=I.permutations(rng, 3, 60))
        w = I.Workload("ties", [s], [I.Instance(0, t, W, p) for t in (5, 30) for W in (1, 4) for p in (-1, 0, 2)])
    elif case in ("k1", "k16"):
        w = I.config(3, n_t=1, S=6, R=150)
        w.k = 1 if case == "k1" else 16
    elif case == "ar1":
        w = I.ar1_analysis("unidirectional", S=4, R=20)
    else:
        w = I.config(5, n_t=1, S=3)
    ds = te.to_device(w.series)
    te.te_set_search(te_handle, False)
    try:
        ref = te.te_estimate(te_handle, ds, w.instances, w.k, want_counts=True)
        ex_pairs, _, swept0 = te.te_last_work(te_handle)
        ex_pass = te.te_last_pass_work(te_handle)
    finally:
        te.te_set_search(te_handle, True)
    got = te.te_estimate(te_handle, ds, w.instances, w.k, want_counts=True)
    sw_pairs, _, swept1 = te.te_last_work(te_handle)
    (p1, p2), (c1, c2) = te.te_last_pass_work(te_handle)
    torch.cuda.synchronize()
    assert not swept0 and swept1
    assert torch.equal(ref["counts"], got["counts"]) and torch.equal(ref["eps"], got["eps"])
    assert torch.max(torch.abs(ref["te"] - got["te"])).item() <= 1e-9
    assert 0 < sw_pairs <= ex_pairs
    # work by pass: N^2 per pass for the exhaustive search; the sweep's two passes add up to its
    # total and both took cycles
    assert ex_pass == ((ex_pairs // 2, ex_pairs // 2), (0, 0))
    assert p1 + p2 == sw_pairs and p1 > 0 and p2 > 0
    assert c1 > 0 and c2 > 0


def test_plan_reuse_follows_the_inputs(te_handle):
    """A call identical to the previous one reuses its plan; a changed instance, series field or
    setting must give a new plan (results of the new inputs, checked against the oracle)."""
    w = I.config(3, n_t=2, S=6, R=120)
    ds = te.to_device(w.series)
    a = te.te_estimate(te_handle, ds, w.instances, w.k).clone()
    b = te.te_estimate(te_handle, ds, w.instances, w.k).clone()
    insts = list(w.instances)
    insts[3] = I.Instance(0, insts[3].t_start, insts[3].window, 5 if insts[3].perm != 5 else 4)
    c = te.te_estimate(te_handle, ds, insts, w.k).clone()
    s2 = w.series[0]
    ds2 = [te.DeviceSeries(ds[0].src, ds[0].tgt, ds[0].d, ds[0].tau, ds[0].u + 1, ds[0].perms)]  # same buffers
    d = te.te_estimate(te_handle, ds2, w.instances, w.k).clone()
    te.te_set_search(te_handle, False)
    try:
        e = te.te_estimate(te_handle, ds, w.instances, w.k).clone()
    finally:
        te.te_set_search(te_handle, True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    o_c = oracle.te_batch(w.series, insts, w.k)
    assert np.max(np.abs(c.cpu().numpy() - o_c)) <= TOL
    su = I.Series(s2.src, s2.tgt, d=s2.d, tau=s2.tau, u=s2.u + 1, perms=s2.perms)
    o_d = oracle.te_batch([su], w.instances, w.k)
    assert np.max(np.abs(d.cpu().numpy() - o_d)) <= TOL
    assert torch.max(torch.abs(a - e)).item() <= 1e-9


@pytest.mark.parametrize("d,R,W,ties", [(1, 1500, 3, False), (1, 2001, 3, True), (2, 1700, 5, False),
                                        (2, 2731, 3, True), (3, 1100, 4, False)])
def test_strip_sweep_equals_exhaustive(te_handle, d, R, W, ties):
    """Resident groups of 4096+ points are cut into strips by a second target coordinate (y_t for
    d = 1, y_{t'-1-tau} for d >= 2), each padded to groups of four: radii and counts must equal the
    exhaustive search exactly (ragged strip sizes, many equal keys, several surrogates)."""
    rng = np.random.default_rng(R + 10 * d)
    if ties:
        src = rng.integers(0, 5, (R, 60)).astype(np.float32)
        tgt = rng.integers(0, 5, (R, 60)).astype(np.float32)
    else:
        src, tgt = I.ar2_pair(rng, R, 60)
    s = I.Series(src, tgt, d=d, tau=2, u=3, perms=I.permutations(rng, 2, R))
    insts = [I.Instance(0, 20, W, p) for p in (-1, 0, 1)]
    ds = te.to_device([s])
    te.te_set_sharing(te_handle, False)
    try:
        te.te_set_search(te_handle, False)
        try:
            ref = te.te_estimate(te_handle, ds, insts, 4, want_counts=True)
        finally:
            te.te_set_search(te_handle, True)
        got = te.te_estimate(te_handle, ds, insts, 4, want_counts=True)
        torch.cuda.synchronize()
        pairs, _, swept = te.te_last_work(te_handle)
    finally:
        te.te_set_sharing(te_handle, True)
    assert swept and pairs < 2 * 3 * (R * W) ** 2
    assert torch.equal(ref["eps"], got["eps"]) and torch.equal(ref["counts"], got["counts"])
    assert torch.max(torch.abs(ref["te"] - got["te"])).item() <= 1e-9
