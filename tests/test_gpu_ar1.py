"""The paper's coupled AR(1) scenarios (Table 1, Eq. 12 - Eq. 16) at the paper's protocol: 50
trials x 3000 samples, analysis windows of 300 samples from 0.2 s, delays scanned over 1..20
(1..30 for the bidirectional scenario), 500 trial-shuffled surrogates per (delay, window), k = 4,
d = 1, tau = 1, both directions (Y -> X by exchanging source and target).

A window counts as significant when the p-value at the reconstructed delay (the delay of largest
TE, Eq. 5) is at most alpha / n_delays (alpha = 0.05, Bonferroni over the scanned delays): with
500 surrogates that is p <= 0.002. Inputs are seeded, so every assertion below is a fixed fact of
these series; each one restates a qualitative result of the paper's AR(1) Results section:
  (1) unidirectional: transfer X -> Y after the onset at 1 s at the true delay 10, none before;
  (2) two-step: no transfer before 1 s, transfer in windows 4 - 8, the true delay 10 after the
      second step at 2 s (windows 7, 8); the paper also reports one false positive Y -> X;
  (3) bidirectional: X -> Y in windows 4 - 8 with delay 10 from window 6 on, Y -> X only after
      2 s (windows 7, 8) with its true delay 20.
Parity: sampled query points of full-size estimates against the CPU oracle, bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_1401_4068_gb300 import inputs as I
from paper_1401_4068_gb300 import te

pytestmark = pytest.mark.gpu
S = 500


def _scan(h, name, direction):
    w = I.ar1_analysis(name, S=S)
    s = w.series[0]
    if direction == "YX":
        s = I.Series(s.tgt, s.src, d=s.d, tau=s.tau, u=s.u, perms=s.perms)
    u_hi = w.extra["u_hi"]
    out = te.te_delay_scan(h, te.to_device([s])[0], w.t_starts[0], w.window, 1, u_hi, w.S, w.k)
    torch.cuda.synchronize()
    te.te_sync_status(h)
    ub = out["u_best"].cpu().numpy()
    p = out["p"].cpu().numpy()
    tev = out["te"].cpu().numpy()
    p_best = np.array([p[ub[j] - 1, j] for j in range(len(ub))])
    te_best = np.array([tev[ub[j] - 1, j] for j in range(len(ub))])
    sig = p_best <= 0.05 / u_hi
    return s, w, ub, sig, te_best


def test_unidirectional_scenario(te_handle):
    _, _, ub, sig, te_best = _scan(te_handle, "unidirectional", "XY")
    assert list(sig) == [False, False, False, True]      # windows from 0.2 s, 0.5 s, 0.8 s, 1.1 s
    assert int(ub[3]) == 10 and abs(int(ub[2]) - 10) <= 2  # the transition window already near 10
    assert te_best[3] > 0.08 and np.max(te_best[:2]) < 0.03
    _, _, _, sig_r, _ = _scan(te_handle, "unidirectional", "YX")
    assert not sig_r.any()                               # no coupling Y -> X


def test_two_step_scenario(te_handle):
    _, _, ub, sig, te_best = _scan(te_handle, "two-step", "XY")
    assert not sig[:3].any()                             # before the first step (0.2 - 1.1 s)
    assert sig[3:].all()                                 # windows 4 - 8 (1.1 - 2.6 s)
    assert int(ub[6]) == 10 and int(ub[7]) == 10         # after the second step: the true delay
    # the second step doubles the coupling: TE in windows 7, 8 well above windows 4 - 6
    assert np.min(te_best[6:]) > 2 * np.max(te_best[3:6])
    _, _, _, sig_r, _ = _scan(te_handle, "two-step", "YX")
    assert sig_r.sum() <= 1                              # no coupling Y -> X (the paper saw one false positive)


def test_bidirectional_scenario(te_handle):
    _, _, ub, sig, te_best = _scan(te_handle, "bidirectional", "XY")
    assert sig[3:].all()                                 # X -> Y from window 4 on
    assert list(ub[5:]) == [10, 10, 10]                  # the true delay from window 6 on
    assert np.min(te_best[3:]) > 3 * np.max(te_best[:2])
    _, _, ub_r, sig_r, te_r = _scan(te_handle, "bidirectional", "YX")
    assert not sig_r[:6].any()                           # Y -> X only after its onset at 2 s
    assert sig_r[6:].all() and list(ub_r[6:]) == [20, 20]
    assert np.min(te_r[6:]) > 3 * np.max(te_r[:6])


@pytest.mark.parametrize("name,direction,window,u", [("bidirectional", "YX", 6, 20), ("two-step", "XY", 4, 4)])
def test_sampled_points_match_the_oracle(te_handle, name, direction, window, u):
    """Full-size estimates of the scenarios (15,000 points): radii and the three counts at 64
    sampled query points equal the oracle's, for the original and two surrogates."""
    w = I.ar1_analysis(name, S=4)
    s = w.series[0]
    if direction == "YX":
        s = I.Series(s.tgt, s.src, d=s.d, tau=s.tau, u=u, perms=s.perms)
    else:
        s = I.Series(s.src, s.tgt, d=s.d, tau=s.tau, u=u, perms=s.perms)
    t0 = w.t_starts[0][window]
    insts = [I.Instance(0, t0, w.window, p) for p in (-1, 0, 3)]
    res = te.te_estimate(te_handle, te.to_device([s]), insts, 4, want_counts=True)
    torch.cuda.synchronize()
    N = s.R * w.window
    eps = res["eps"].cpu().numpy().reshape(len(insts), N)
    counts = res["counts"].cpu().numpy().reshape(len(insts), 3, N)
    q = np.random.default_rng(7 + window).choice(N, 64, replace=False)
    for j, it in enumerate(insts):
        pts = oracle.embed(s.src, s.tgt, s.d, s.tau, s.u, it.t_start, it.window,
                           None if it.perm < 0 else s.perms[it.perm])
        o_eps, o_counts = oracle.points_at(pts, 1, 1, 4, q)
        np.testing.assert_array_equal(eps[j, q], o_eps)
        np.testing.assert_array_equal(counts[j][:, q], o_counts)
