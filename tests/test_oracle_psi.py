"""Pins of the oracle's digamma (the nonlinearity of Eq. 9) against values that do not come
from the oracle: Euler's constant, a hand-summed harmonic number, scipy's digamma and the
asymptotic expansion."""
import math

import numpy as np
import pytest
from scipy.special import digamma as sp_digamma

import oracle

EULER_GAMMA = 0.5772156649015329


def test_psi_1_is_minus_euler_gamma():
    assert oracle.digamma(1) == pytest.approx(-EULER_GAMMA, abs=1e-16)


def test_psi_4_hand_value():
    # psi(4) = 1 + 1/2 + 1/3 - gamma
    assert oracle.digamma(4) == pytest.approx(1.2561176684318005, abs=2e-16)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 10, 57, 100, 1001, 4096, 12001, 20000])
def test_psi_matches_scipy(n):
    assert oracle.digamma(n) == pytest.approx(float(sp_digamma(n)), abs=1e-11)


def test_psi_asymptotic_at_1e4():
    n = 10_000
    asym = math.log(n) - 1 / (2 * n) - 1 / (12 * n ** 2) + 1 / (120 * n ** 4)
    assert abs(oracle.digamma(n) - asym) < 1e-12


def test_psi_invalid():
    assert math.isnan(oracle.digamma(0))
