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


# ---- coupled Lorenz systems (Eq. 11)
def test_lorenz_attractor_statistics():
    """Uncoupled, each system is the classic Lorenz attractor (sigma 10, rho 28, beta 8/3), whose
    y coordinate (V here) has mean 0 by symmetry and a standard deviation of about 9.0."""
    rng = np.random.default_rng(3)
    x, y = I.lorenz_pair(rng, 40, 3000, gamma=0.0)
    for v in (x, y):
        assert np.isfinite(v).all()
        assert abs(float(v.mean())) < 0.6
        assert 8.6 < float(v.std()) < 9.4


def test_lorenz_coupling_is_unidirectional_and_windowed():
    """X never depends on Y; Y is unchanged before the coupling interval and changed inside it."""
    a = I.lorenz_pair(np.random.default_rng(4), 6, 1500, coupled=(1000, 2000))
    b = I.lorenz_pair(np.random.default_rng(4), 6, 1500, gamma=0.0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1][:, :1000], b[1][:, :1000])
    assert np.abs(a[1][:, 1100:] - b[1][:, 1100:]).max() > 1.0


def test_lorenz_coupling_delay():
    """V_X(t - delta)^2 drives dV_Y/dt: its correlation with the increments of V_Y peaks near the
    coupling delay (45 samples) and is small far from it."""
    x, y = I.lorenz_pair(np.random.default_rng(5), 40, 1200, coupled=None)
    dy = np.diff(y.astype(np.float64), axis=1)
    corr = {}
    for lag in range(20, 71, 2):
        xs = x[:, 200 - lag:1100 - lag].astype(np.float64) ** 2
        corr[lag] = np.corrcoef(xs.ravel(), dy[:, 200:1100].ravel())[0, 1]
    best = max(corr, key=corr.get)
    assert 38 <= best <= 46, corr
    assert corr[best] > 0.3 and corr[20] < 0.2


def test_lorenz_integrator_converges():
    """Fourth-order convergence of the RK4 grid over a short horizon (before chaos amplifies the
    differences): halving the step shrinks the error against a 16-step-per-sample solution by
    about 2^4, and 4 steps per sample are already far below the signal scale."""
    kw = dict(burn=0, coupled=None)
    a = I.lorenz_pair(np.random.default_rng(6), 4, 40, substeps=4, **kw)
    b = I.lorenz_pair(np.random.default_rng(6), 4, 40, substeps=8, **kw)
    ref = I.lorenz_pair(np.random.default_rng(6), 4, 40, substeps=16, **kw)
    e4 = max(np.abs(a[i].astype(np.float64) - ref[i]).max() for i in (0, 1))
    e8 = max(np.abs(b[i].astype(np.float64) - ref[i]).max() for i in (0, 1))
    assert e4 < 2e-4
    assert e4 / e8 > 8


def test_lorenz_workload_shapes():
    w = I.lorenz_analysis(S=3, R=8, T=3000)
    assert w.t_starts == [[200, 1600, 2750]] and w.window == 250
    assert (w.extra["u_lo"], w.extra["u_hi"]) == (35, 55)
    assert len(w.instances) == 3 * 4 and w.n_points(w.instances[0]) == 8 * 250
    rob = I.lorenz_robustness(S=2, R=12, trials=(3, 10))
    assert sorted(rob) == [600, 2000]
    assert rob[2000].n_points(rob[2000].instances[0]) == 2000
    c = I.paper_chunk(chunks=3)
    assert len(c.instances) == 3
    assert c.n_points(c.instances[0]) == 30094 and c.joint_dim(c.instances[0]) == 17
