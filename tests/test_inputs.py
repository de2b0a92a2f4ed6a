"""The seeded input generators: shapes, determinism, and the Table 1 / Eq. 14 - Eq. 16 coupling
ramps of the AR(1) scenarios (values typed by hand from the equations)."""
import math

import numpy as np
import pytest

from paper_1401_4068_gb300 import inputs as I


def test_configs_have_the_stated_shapes():
    shapes = {1: (1, 1000, 5), 2: (100, 1500, 7)}
    for cid, (n, N, D) in shapes.items():
        w = I.config(cid)
        assert len(w.instances) == n
        assert {w.n_points(i) for i in w.instances} == {N}
        assert {w.joint_dim(i) for i in w.instances} == {D}
    w3 = I.config(3, n_t=2, S=4)
    assert len(w3.instances) == 2 * 5 and w3.n_points(w3.instances[0]) == 1200


def test_generators_are_deterministic():
    a = I.config(3, n_t=1, S=3)
    b = I.config(3, n_t=1, S=3)
    np.testing.assert_array_equal(a.series[0].src, b.series[0].src)
    np.testing.assert_array_equal(a.series[0].perms, b.series[0].perms)


def test_permutations_are_permutations():
    p = I.permutations(np.random.default_rng(0), 7, 40)
    assert p.dtype == np.int32
    for row in p:
        assert sorted(row.tolist()) == list(range(40))


def test_table1_parameters():
    assert I.AR1_SCENARIOS["unidirectional"] == dict(ax=0.75, ay=0.35, byx=0.0, bxy=-0.35, dyx=0, dxy=10)
    assert I.AR1_SCENARIOS["bidirectional"]["ax"] == 0.475
    assert I.AR1_SCENARIOS["bidirectional"]["dyx"] == 20


def test_coupling_ramps():
    t = np.array([0.0, 1000.0, 2000.0, 3000.0])
    gxy, gyx = I.ar1_couplings("unidirectional", t)
    # gamma_XY = -0.35 * 0.5 * (1 + tanh(0.05 (t - 1000)))
    assert gxy[1] == pytest.approx(-0.35 * 0.5)
    assert gxy[0] == pytest.approx(-0.35 * 0.5 * (1 + math.tanh(-50.0)))
    assert gxy[3] == pytest.approx(-0.35)
    assert np.all(gyx == 0)
    g2, _ = I.ar1_couplings("two-step", t)
    assert g2[1] == pytest.approx(-0.35 * 0.5 * 0.5 * (1 + (1 + math.tanh(-50.0))))
    assert g2[3] == pytest.approx(-0.35)
    _, gb = I.ar1_couplings("bidirectional", t)
    assert gb[2] == pytest.approx(-0.4 * 0.5)


def test_ar1_scenario_shapes():
    x, y = I.ar1_scenario(np.random.default_rng(1), "bidirectional", R=4, T=500)
    assert x.shape == (4, 500) and y.dtype == np.float32
    w = I.ar1_analysis("unidirectional", S=3, R=5)
    assert w.t_starts[0] == [200, 500, 800, 1100] and w.window == 300
