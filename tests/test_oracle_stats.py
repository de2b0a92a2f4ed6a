"""Statistical pins of the oracle: values fixed by mathematics, not by the oracle.

  * Mutual-information special case: with an empty conditioning group the estimator of Eq. 9
    reduces to the KSG mutual-information estimator (n_y- = N-1 for every point), whose
    target for a bivariate Gaussian is -1/2 ln(1 - rho^2).
  * Closed form of linear Gaussian processes: TE = 1/2 ln of the conditional-variance ratio
    (the TE / linear Granger-causality equivalence the paper cites).
  * TE near zero without coupling, and trial-shuffled surrogates near zero with the original
    estimate above all of them (the surrogate test of the paper).
Tolerances: 3 standard errors of the mean over independent estimates plus 0.02 nats of
finite-sample bias allowance for k = 4 at these point counts."""
import numpy as np
import pytest

import oracle
from closed_form import gaussian_mi, gaussian_te
from paper_1401_4068_gb300 import inputs as I


def _mean_se(v):
    v = np.asarray(v)
    return v.mean(), v.std(ddof=1) / np.sqrt(len(v))


def test_mi_special_case_bivariate_gaussian():
    rho = 0.6
    vals = []
    for seed in range(8):
        x, y = I.gaussian_pair_iid(np.random.default_rng(100 + seed), 1, 1500, rho)
        pts = np.stack([y[0], x[0]], axis=1)  # [y_t | (empty y-) | x-]
        te, _, c = oracle.te_points(pts, 0, 1, 4)
        assert np.all(c[0] == 1500 - 1)  # empty conditioning space: every point counted
        vals.append(te)
    m, se = _mean_se(vals)
    assert abs(m - gaussian_mi(rho)) < 3 * se + 0.02


def test_ar2_closed_form_c1_shape():
    w = I.config(1)
    s = w.series[0]
    tes = [oracle.te_points(oracle.embed(s.src, s.tgt, 2, 1, 5, t, 5), 2, 2, 4)[0]
           for t in range(20, 290, 14)]
    m, se = _mean_se(tes)
    truth = gaussian_te(I.AR_AX, I.AR_AY, I.AR_COUPLING, I.AR_U, d=2, tau=1, u=5)
    assert 0.12 < truth < 0.14
    assert abs(m - truth) < 3 * se + 0.02


def test_uncoupled_te_near_zero():
    rng = np.random.default_rng(11)
    src, tgt = I.ar2_pair(rng, 200, 300, coupling_start=None)
    tes = [oracle.te_points(oracle.embed(src, tgt, 2, 1, 5, t, 5), 2, 2, 4)[0]
           for t in range(20, 290, 27)]
    m, se = _mean_se(tes)
    assert abs(m) < 3 * se + 0.02
    assert gaussian_te(I.AR_AX, I.AR_AY, 0.0, I.AR_U, d=2, tau=1, u=5) == pytest.approx(0, abs=1e-12)


def test_surrogates_near_zero_and_original_significant():
    w = I.config(1)
    s = w.series[0]
    S = 24
    s.perms = I.permutations(np.random.default_rng(5), S, s.R)
    insts = [I.Instance(0, 100, 5, -1)] + [I.Instance(0, 100, 5, p) for p in range(S)]
    te = oracle.te_batch([s], insts, 4)
    te0, ts = te[0], te[1:]
    assert oracle.pvalue(te0, ts) == 0.0
    m, se = _mean_se(ts)
    assert abs(m) < 3 * se + 0.02
    assert te0 > 0.08
    # identity surrogate reproduces the original exactly
    s.perms = np.arange(s.R, dtype=np.int32)[None, :]
    te_id = oracle.te_batch([s], [I.Instance(0, 100, 5, 0)], 4)
    assert te_id[0] == te0


def test_pvalue_definition():
    assert oracle.pvalue(0.5, np.array([0.1, 0.5, 0.7, 0.2])) == 0.5
    assert oracle.pvalue(1.0, np.array([0.1, 0.2])) == 0.0
