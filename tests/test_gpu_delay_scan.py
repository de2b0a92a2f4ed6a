"""Delay reconstruction (Eq. 5, "Reconstruction of information transfer delays") through
te_delay_scan: every (u, t, surrogate) estimate against the oracle (TE within 1e-6, p-values
equal), the reconstructed delay against the oracle's argmax and against the true coupling
delay, and argument errors. The paper's AR(1) scenarios at full protocol are in
tests/test_gpu_ar1.py."""
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
