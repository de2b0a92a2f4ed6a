"""Delay reconstruction (Eq. 5, "Reconstruction of information transfer delays") through
te_delay_scan: every (u, t, surrogate) estimate against the oracle (TE within 1e-6, p-values
equal), the reconstructed delay against the oracle's argmax and against the true coupling
delay, and the qualitative detection results of the paper's unidirectional AR(1) scenario
(Table 1, Eq. 12 - Eq. 15): no transfer before the coupling onset, transfer near the true
delay of 10 samples after it."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu
TOL = 1e-6


def _oracle_scan(s, t_starts, window, u_lo, u_hi, S, k):
    series = [dataclasses.replace(s, u=u) for u in range(u_lo, u_hi + 1)]
    insts = [I.Instance(iu, t, window, m) for iu in range(len(series)) for t in t_starts for m in range(-1, S)]
    te_all = oracle.te_batch(series, insts, k).reshape(len(series), len(t_starts), S + 1)
    return te_all


def test_delay_scan_matches_oracle_and_recovers_the_delay(te_handle):
    w = I.config(1)
    s = dataclasses.replace(w.series[0], d=1)
    s.perms = I.permutations(np.random.default_rng(21), 8, s.R)
    ts, W, S, k = [20, 110, 230], 5, 8, 4
    ds = te.to_device([s])[0]
    out = te.te_delay_scan(te_handle, ds, ts, W, 1, 9, S, k)
    torch.cuda.synchronize()
    o = _oracle_scan(s, ts, W, 1, 9, S, k)
    g_te = out["te"].cpu().numpy()
    assert np.max(np.abs(g_te - o[:, :, 0])) <= TOL
    for iu in range(o.shape[0]):
        for j in range(len(ts)):
            assert np.min(np.abs(o[iu, j, 1:] - o[iu, j, 0])) > 2 * TOL
            assert out["p"][iu, j].item() == oracle.pvalue(o[iu, j, 0], o[iu, j, 1:])
    ub = out["u_best"].cpu().numpy()
    np.testing.assert_array_equal(ub, 1 + np.argmax(o[:, :, 0], axis=0))
    # closed form: TE(u) of this pair with d = 1 peaks at the true delay u = 5 (0.136 vs <= 0.022)
    assert np.all(ub == I.AR_U)


def test_delay_scan_argument_errors(te_handle):
    w = I.config(1)
    ds = te.to_device(w.series)[0]
    with pytest.raises(te.TEError, match="TE_ERANGE"):
        te.te_delay_scan(te_handle, ds, [10], 5, 1, 12, 0, 4)   # u = 12 reaches before sample 0
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_delay_scan(te_handle, ds, [100], 5, 5, 3, 0, 4)   # empty u range
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_delay_scan(te_handle, ds, [100], 5, 1, 3, 4, 4)   # no permutations for S = 4


def test_ar1_unidirectional_scenario_detection(te_handle):
    # 50 trials x 3000 samples, windows of 300 samples at 0.2, 0.5, 0.8 and 1.1 s, u = 1..20,
    # 100 surrogates per (u, window); coupling X -> Y ramps up around 1.0 s with delay 10.
    # p-values are per (u, window), uncorrected for the 20 scanned delays.
    w = I.ar1_analysis("unidirectional", S=100)
    ds = te.to_device(w.series)[0]
    out = te.te_delay_scan(te_handle, ds, w.t_starts[0], w.window, 1, 20, w.S, w.k)
    torch.cuda.synchronize()
    p = out["p"].cpu().numpy()       # [u - 1][window]
    ub = out["u_best"].cpu().numpy()
    tev = out["te"].cpu().numpy()
    # before the onset (0.2-0.5 s, 0.5-0.8 s): TE near zero for every delay and no more
    # uncorrected detections than the 5 % level allows for
    assert np.max(tev[:, :2]) < 0.03
    assert np.mean(p[:, :2] < 0.05) <= 0.15
    # after the onset (1.1-1.4 s): significant transfer, the TE profile over u peaks at the
    # true delay (closed form 0.104 at u = 10 vs 0.051 / 0.047 at 9 / 11)
    assert int(ub[3]) == 10 and p[ub[3] - 1, 3] == 0.0
    assert tev[10 - 1, 3] > 0.08
    assert np.all(np.delete(tev[:, 3], 10 - 1) < tev[10 - 1, 3] - 0.03)
    # during the transition (0.8-1.1 s) the reconstructed delay is already near 10
    assert abs(int(ub[2]) - 10) <= 2
