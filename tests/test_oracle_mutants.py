"""The pins must catch plausible mistakes in the oracle.

Each case below plants one mistake (a dropped term, a wrong sign, an off-by-one index, a
non-strict comparison, a transposed operand ...) into a temporary copy of the oracle's C
source, builds it on the CPU and runs the pins against it.  Every mutant must fail at least
one pin.  Nothing here touches the library or a GPU."""
import ctypes as C
import json
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.special import digamma as sp_digamma

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "te_oracle.c")
HDR = os.path.join(os.path.dirname(HERE), "oracle", "te_oracle.h")

MUTANTS = [
    ("non-strict count", "< e) ++nz", "<= e) ++nz"),
    ("wrong digamma sign", "- psi[c[(size_t)N + i] + 1]", "+ psi[c[(size_t)N + i] + 1]"),
    ("dropped digamma term", " - psi[c[(size_t)2 * N + i] + 1]", ""),
    ("eps off by one", "*eps_i = a[k - 1].dist", "*eps_i = a[k > 1 ? k - 2 : 0].dist"),
    ("self counted in the range counts", "        if (j == i) continue;\n        const float* pj",
     "        const float* pj"),
    ("target past index", "y[t - 1 - m * tau]", "y[t - m * tau]"),
    ("source delay index", "x[t - u - m * tau]", "x[t - u + 1 - m * tau]"),
    ("digamma recurrence", "t[n + 1] = t[n] + 1.0 / (double)n", "t[n + 1] = t[n] + 1.0 / (double)(n + 1)"),
    ("joint space used for n_xz", "maxnorm(pi, pj, 1, D) < e) ++nxz", "maxnorm(pi, pj, 0, D) < e) ++nxz"),
    ("y_t dropped from n_yz", "maxnorm(pi, pj, 0, 1 + dy) < e) ++nyz", "maxnorm(pi, pj, 0, 1) < e) ++nyz"),
    ("average over N-1", "sum / (double)N", "sum / (double)(N - 1)"),
    ("psi(k) dropped", "*te = psi[k] + sum", "*te = sum"),
    ("p-value strict", "if (te_surr[s] >= te_orig)", "if (te_surr[s] > te_orig)"),
    ("neighbour tie order", "(a->j > b->j) - (a->j < b->j)", "(a->j < b->j) - (a->j > b->j)"),
    ("permutation on the target", "const float* y = tgt + (size_t)r * T;",
     "const float* y = tgt + (size_t)rs * T;"),
    ("transposed difference operand", "fabsf(a[c] - b[c])", "fabsf(a[c] - b[c - (c > 0)])"),
    ("surrogate row of the permutation table", "perm = s->perms + (size_t)in->perm * s->R;",
     "perm = s->perms + (size_t)in->perm;"),
    ("wrong series of an instance", "const oracle_series* s = &jb->series[in->series];",
     "const oracle_series* s = &jb->series[0];"),
    ("counts block offset", "jb->counts + 3 * jb->off[i]", "jb->counts + jb->off[i]"),
    ("point offsets from the first series", "off[i] + (int64_t)series[inst[i].series].R * inst[i].window",
     "off[i] + (int64_t)series[0].R * inst[i].window"),
    ("surrogate pairing on the original", "if (in->perm >= 0) {", "if (in->perm > 0) {"),
]


def _run_pins(lib) -> list:
    """Run the deterministic pins against a loaded oracle build; return the failures."""
    saved = oracle._lib
    oracle._lib = lib
    fails = []
    try:
        g = json.load(open(os.path.join(HERE, "golden", "worked_example.json")))
        pts = np.array(g["points"], np.float32)
        for case in g["cases"]:
            eps, nn = oracle.knn(pts, case["k"], want_nn=True)
            if not np.array_equal(eps, case["eps"]): fails.append("eps")
            if not np.array_equal(nn, case["nn"]): fails.append("nn")
            c = oracle.range_count(pts, 1, 1, np.array(case["eps"], np.float32))
            if not np.array_equal(c, [case["n_z"], case["n_yz"], case["n_xz"]]): fails.append("counts")
            te, _, _ = oracle.te_points(pts, 1, 1, case["k"])
            if abs(te - case["te"]) > 1e-12: fails.append("te")
        ge = json.load(open(os.path.join(HERE, "golden", "embedding_ramp.json")))
        R, T = ge["R"], ge["T"]
        src = np.array([[10000 * r + t for t in range(T)] for r in range(R)], np.float32)
        for case in ge["cases"]:
            if "points" not in case:
                continue
            perm = None if case["perm"] is None else np.array(case["perm"], np.int32)
            try:
                p = oracle.embed(src, src + 5000, case["d"], case["tau"], case["u"],
                                 case["t_start"], case["window"], perm)
                if not np.array_equal(p, case["points"]): fails.append("embed")
            except (IndexError, ValueError):
                fails.append("embed-error")
        for n, v in ((1, -0.5772156649015329), (4, 1.2561176684318005), (1001, sp_digamma(1001))):
            if abs(oracle.digamma(n) - v) > 1e-11: fails.append("digamma")
        # oracle.digamma evaluates psi directly; Eq. 9 goes through the table: check both
        pts1 = np.array([[0, 0, 0], [1, 0, 0], [0, 2, 0], [0, 0, 3], [5, 5, 5], [2, 2, 9]], np.float32)
        te, _, c = oracle.te_points(pts1, 1, 1, 2)
        ref = sp_digamma(2) + np.mean(sp_digamma(c[0] + 1) - sp_digamma(c[1] + 1) - sp_digamma(c[2] + 1))
        if abs(te - ref) > 1e-12: fails.append("te-table")
        if oracle.pvalue(0.5, np.array([0.1, 0.5, 0.7, 0.2])) != 0.5: fails.append("pvalue")
        fails += batch_dispatch_failures()
    finally:
        oracle._lib = saved
    return fails


def batch_dispatch_failures() -> list:
    """te_batch against physically shuffled trials (Fig. 3: a surrogate pairs the target's
    repetitions with reordered source repetitions).  Two series of different trial counts and
    delays, instances in mixed order with different windows; for each one the expected values
    come from the source array whose rows were reordered with numpy (row r of the surrogate's
    source = source row perm[r]) and analysed as an original, so no permutation offset, series
    index or output offset of the batch code is involved."""
    fails = []
    rng = np.random.default_rng(20140728)
    Ser = type("Ser", (), {})
    series = []
    for R, T, d, u in ((5, 30, 1, 2), (6, 28, 2, 3)):
        s = Ser()
        s.src = rng.standard_normal((R, T)).astype(np.float32)
        s.tgt = rng.standard_normal((R, T)).astype(np.float32)
        s.d, s.tau, s.u = d, 1, u
        s.perms = np.stack([rng.permutation(R) for _ in range(3)]).astype(np.int32)
        series.append(s)
    Inst = type("Inst", (), {})
    spec = [(1, 9, 3, 2), (0, 8, 4, -1), (0, 12, 3, 0), (1, 9, 3, 1), (0, 8, 4, 2), (1, 14, 5, -1), (0, 8, 4, 1)]
    insts = []
    for si, t, W, p in spec:
        it = Inst()
        it.series, it.t_start, it.window, it.perm = si, t, W, p
        insts.append(it)
    k = 2
    te, counts, eps = oracle.te_batch(series, insts, k, n_threads=2, want_counts=True)
    off = 0
    for i, it in enumerate(insts):
        s = series[it.series]
        src = s.src if it.perm < 0 else s.src[s.perms[it.perm]]
        pts = oracle.embed(src, s.tgt, s.d, s.tau, s.u, it.t_start, it.window, None)
        N = pts.shape[0]
        te_i, eps_i, c_i = oracle.te_points(pts, s.d, s.d, k)
        if te[i] != te_i: fails.append(f"batch-te[{i}]")
        if not np.array_equal(counts[3 * off:3 * (off + N)].reshape(3, N), c_i): fails.append(f"batch-counts[{i}]")
        if not np.array_equal(eps[off:off + N], eps_i): fails.append(f"batch-eps[{i}]")
        off += N
    if off != eps.shape[0]: fails.append("batch-size")
    return fails


def test_batch_dispatch_pin():
    assert batch_dispatch_failures() == []


def _build(tmp_path, find, repl):
    s = open(SRC).read()
    assert s.count(find) >= 1, find
    s = s.replace(find, repl, 1)
    d = tmp_path / "m"
    d.mkdir()
    shutil.copy(HDR, d / "te_oracle.h")
    (d / "te_oracle.c").write_text(s)
    so = d / "liboracle_mutant.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(so), str(d / "te_oracle.c"), "-lm"], check=True)
    return oracle.configure(C.CDLL(str(so)))


def test_pins_pass_on_the_real_oracle():
    assert _run_pins(oracle._load()) == []


@pytest.mark.parametrize("name,find,repl", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, find, repl):
    lib = _build(tmp_path, find, repl)
    assert _run_pins(lib), f"planted mistake '{name}' passed every pin"
