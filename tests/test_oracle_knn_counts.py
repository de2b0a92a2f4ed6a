"""Pins of the oracle's kNN search, range counts and digamma sum (Eq. 9 / Eq. 10 with the
maximum norm of the paper's search) against values the oracle does not produce:
  * a hand-worked example with a tie exactly at eps (tests/golden/worked_example.json);
  * exhaustive enumeration on tiny integer inputs, in exact integer arithmetic, with eps and
    the neighbour list defined by counting instead of sorting, and scipy's digamma;
  * exact invariants of the definition (point order, power-of-two scaling, coordinate order
    inside a marginal group, projection order relations)."""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.special import digamma as sp_digamma

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "worked_example.json")))


@pytest.mark.parametrize("case", GOLD["cases"])
def test_worked_example(case):
    pts = np.array(GOLD["points"], np.float32)
    k = case["k"]
    eps, nn = oracle.knn(pts, k, want_nn=True)
    np.testing.assert_array_equal(eps, np.array(case["eps"], np.float32))
    np.testing.assert_array_equal(nn, np.array(case["nn"], np.int32))
    counts = oracle.range_count(pts, GOLD["dy"], GOLD["dx"], eps)
    np.testing.assert_array_equal(counts[0], case["n_z"])
    np.testing.assert_array_equal(counts[1], case["n_yz"])
    np.testing.assert_array_equal(counts[2], case["n_xz"])
    te, _, _ = oracle.te_points(pts, GOLD["dy"], GOLD["dx"], k)
    assert te == pytest.approx(case["te"], abs=1e-14)


# ---------------------------------------------------------------- exhaustive enumeration
def _enumerate(P, dy, dx, k):
    """Exact integer KSG quantities by counting (no sorting)."""
    N, D = len(P), len(P[0])

    def dist(i, j, cs):
        return max([abs(P[i][c] - P[j][c]) for c in cs], default=0)

    joint = list(range(D))
    eps, nn, cnt = [], [], [[], [], []]
    for i in range(N):
        others = [j for j in range(N) if j != i]
        ds = {j: dist(i, j, joint) for j in others}
        # eps: smallest distance value v with at least k others at distance <= v
        e = min(v for v in ds.values() if sum(1 for j in others if ds[j] <= v) >= k)
        # j is a neighbour iff fewer than k others precede it in (distance, index) order
        nb = sorted(j for j in others
                    if sum(1 for jj in others if (ds[jj], jj) < (ds[j], j)) < k)
        nb.sort(key=lambda j: (ds[j], j))
        eps.append(e)
        nn.append(nb)
        B = list(range(1, 1 + dy))
        A_B = list(range(0, 1 + dy))
        B_C = list(range(1, D))
        cnt[0].append(sum(1 for j in others if dist(i, j, B) < e))
        cnt[1].append(sum(1 for j in others if dist(i, j, A_B) < e))
        cnt[2].append(sum(1 for j in others if dist(i, j, B_C) < e))
    te = float(sp_digamma(k)) + np.mean(
        [sp_digamma(cnt[0][i] + 1) - sp_digamma(cnt[1][i] + 1) - sp_digamma(cnt[2][i] + 1)
         for i in range(N)])
    return eps, nn, cnt, te


CASES = []
rng = np.random.default_rng(7)
for N in (2, 3, 4, 5, 6, 8):
    for (dy, dx) in ((1, 1), (2, 1), (1, 2), (2, 2), (0, 1), (3, 0)):
        for k in sorted({1, N // 2, N - 1}):
            if k >= 1 and N >= k + 1:
                CASES.append((N, dy, dx, k, int(rng.integers(1 << 30))))


@pytest.mark.parametrize("N,dy,dx,k,seed", CASES)
def test_exhaustive_small_integer(N, dy, dx, k, seed):
    r = np.random.default_rng(seed)
    D = 1 + dy + dx
    P = r.integers(0, 4, size=(N, D))  # few values: many exact ties
    eps, nn, cnt, te = _enumerate(P.tolist(), dy, dx, k)
    pts = P.astype(np.float32)
    o_eps, o_nn = oracle.knn(pts, k, want_nn=True)
    np.testing.assert_array_equal(o_eps, np.array(eps, np.float32))
    np.testing.assert_array_equal(o_nn, np.array(nn, np.int32))
    o_cnt = oracle.range_count(pts, dy, dx, o_eps)
    np.testing.assert_array_equal(o_cnt, np.array(cnt, np.int32))
    o_te, _, _ = oracle.te_points(pts, dy, dx, k)
    assert o_te == pytest.approx(te, abs=1e-12)


# ---------------------------------------------------------------- invariants
def _rand_points(n, dy, dx, seed):
    return np.random.default_rng(seed).standard_normal((n, 1 + dy + dx)).astype(np.float32)


def test_point_order_invariance():
    pts = _rand_points(80, 2, 2, 1)
    te, eps, c = oracle.te_points(pts, 2, 2, 4)
    perm = np.random.default_rng(2).permutation(80)
    te2, eps2, c2 = oracle.te_points(pts[perm], 2, 2, 4)
    np.testing.assert_array_equal(eps2, eps[perm])
    np.testing.assert_array_equal(c2, c[:, perm])
    assert te2 == pytest.approx(te, abs=1e-12)


@pytest.mark.parametrize("m", [-3, 5])
def test_power_of_two_scaling(m):
    pts = _rand_points(70, 1, 3, 3)
    te, eps, c = oracle.te_points(pts, 1, 3, 3)
    te2, eps2, c2 = oracle.te_points(pts * np.float32(2.0 ** m), 1, 3, 3)
    np.testing.assert_array_equal(eps2, eps * np.float32(2.0 ** m))
    np.testing.assert_array_equal(c2, c)
    assert te2 == te


def test_coordinate_order_inside_groups():
    pts = _rand_points(60, 3, 3, 4)
    te, eps, c = oracle.te_points(pts, 3, 3, 4)
    cols = [0, 3, 1, 2, 6, 4, 5]  # B and C coordinates shuffled inside their groups
    te2, eps2, c2 = oracle.te_points(np.ascontiguousarray(pts[:, cols]), 3, 3, 4)
    np.testing.assert_array_equal(eps2, eps)
    np.testing.assert_array_equal(c2, c)
    assert te2 == te


def test_projection_order_relations():
    pts = _rand_points(200, 2, 2, 5)
    k = 4
    te, eps, c = oracle.te_points(pts, 2, 2, k)
    nz, nyz, nxz = c
    assert np.all(nz >= nyz) and np.all(nz >= nxz)
    # with continuous data there are no ties at eps: exactly k-1 joint neighbours inside
    assert np.all(nyz >= k - 1) and np.all(nxz >= k - 1)


def test_invalid_sizes():
    pts = _rand_points(4, 1, 1, 6)
    with pytest.raises(ValueError):
        oracle.knn(pts, 4)


def test_points_at_equals_the_whole_set_evaluation():
    """The sampled-query entry (used on point sets too large to evaluate whole) gives exactly
    the radii and counts of the full evaluation at the chosen points, ties included."""
    rng = np.random.default_rng(12)
    for pts, dy, dx in ((rng.standard_normal((400, 7)).astype(np.float32), 3, 3),
                        (rng.integers(0, 3, (150, 5)).astype(np.float32), 2, 2)):
        eps = oracle.knn(pts, 4)
        c = oracle.range_count(pts, dy, dx, eps)
        idx = [0, 1, 77, len(pts) - 1, 42]
        e2, c2 = oracle.points_at(pts, dy, dx, 4, idx)
        np.testing.assert_array_equal(e2, eps[idx])
        np.testing.assert_array_equal(c2, c[:, idx])
