"""Pins of the oracle's delay embedding (Eq. 6, Eq. 7, source at t-u, Eq. 10 point order)
against hand-typed coordinates of ramp series (tests/golden/embedding_ramp.json)."""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "embedding_ramp.json")))


def _ramp():
    R, T = GOLD["R"], GOLD["T"]
    src = np.array([[10000 * r + t for t in range(T)] for r in range(R)], np.float32)
    return src, src + np.float32(5000)


@pytest.mark.parametrize("case", GOLD["cases"])
def test_embedding_matches_hand_values(case):
    src, tgt = _ramp()
    perm = None if case["perm"] is None else np.array(case["perm"], np.int32)
    pts = oracle.embed(src, tgt, case["d"], case["tau"], case["u"], case["t_start"],
                       case["window"], perm)
    assert pts.shape == (GOLD["R"] * case["window"], 1 + 2 * case["d"])
    if "points" in case:
        np.testing.assert_array_equal(pts, np.array(case["points"], np.float32))
    else:
        first, last = case["points_first_last"]
        np.testing.assert_array_equal(pts[0], np.array(first, np.float32))
        np.testing.assert_array_equal(pts[-1], np.array(last, np.float32))


@pytest.mark.parametrize("case", GOLD["range_errors"])
def test_embedding_range_errors(case):
    src, tgt = _ramp()
    with pytest.raises(IndexError):
        oracle.embed(src, tgt, case["d"], case["tau"], case["u"], case["t_start"], case["window"])


def test_identity_perm_equals_original():
    src, tgt = _ramp()
    a = oracle.embed(src, tgt, 2, 2, 3, 10, 4)
    b = oracle.embed(src, tgt, 2, 2, 3, 10, 4, perm=np.arange(GOLD["R"], dtype=np.int32))
    np.testing.assert_array_equal(a, b)


def test_bad_perm_rejected():
    src, tgt = _ramp()
    with pytest.raises(ValueError):
        oracle.embed(src, tgt, 1, 1, 1, 5, 1, perm=np.array([0, 1, 3], np.int32))
