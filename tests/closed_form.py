"""Closed-form transfer entropy of linear Gaussian processes (test-side pin of the oracle).

For jointly Gaussian variables TE equals half the log ratio of conditional variances (the
TE / linear Granger-causality equivalence the paper relies on in its discussion of linear
Granger causality):

    TE = 1/2 * ln( Var(y_t | y-) / Var(y_t | y-, x-) ).

The stationary covariance of the coupled AR pair comes from its companion form
s_t = A s_{t-1} + noise via the discrete Lyapunov equation (scipy), and the conditional
variances from the Gaussian conditioning formula.  Nothing here shares code with the oracle.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_discrete_lyapunov


def ar_pair_covariance(ax, ay, coupling, u_true, L, sigma=1.0):
    """Stationary covariance of s_t = [x_t .. x_{t-L+1}, y_t .. y_{t-L+1}] for
    x_t = sum_i ax[i] x_{t-1-i} + e_x,  y_t = sum_i ay[i] y_{t-1-i} + coupling x_{t-u_true} + e_y."""
    n = 2 * L
    A = np.zeros((n, n))
    for i, a in enumerate(ax):
        A[0, i] = a
    for m in range(1, L):
        A[m, m - 1] = 1.0
    for i, a in enumerate(ay):
        A[L, L + i] = a
    # x_{t-u_true} = s_{t-1}[u_true - 1]
    A[L, u_true - 1] += coupling
    for m in range(1, L):
        A[L + m, L + m - 1] = 1.0
    Q = np.zeros((n, n))
    Q[0, 0] = sigma ** 2
    Q[L, L] = sigma ** 2
    return solve_discrete_lyapunov(A, Q)


def _cond_var(S, i, idx):
    if len(idx) == 0:
        return S[i, i]
    Szz = S[np.ix_(idx, idx)]
    Syz = S[i, idx]
    return S[i, i] - Syz @ np.linalg.solve(Szz, Syz)


def gaussian_te(ax, ay, coupling, u_true, d, tau, u, sigma=1.0):
    """Closed-form TE(X -> Y) with target past (y_{t-1}, ..., y_{t-1-(d-1)tau}) and source past
    (x_{t-u}, ..., x_{t-u-(d-1)tau})."""
    L = max(1 + (d - 1) * tau, u + (d - 1) * tau, u_true, len(ax), len(ay)) + 2
    S = ar_pair_covariance(ax, ay, coupling, u_true, L, sigma)
    iy = L  # y_t
    ypast = [L + 1 + m * tau for m in range(d)]
    xpast = [u + m * tau for m in range(d)]
    v1 = _cond_var(S, iy, ypast)
    v2 = _cond_var(S, iy, ypast + xpast)
    return 0.5 * np.log(v1 / v2)


def gaussian_mi(rho):
    """Mutual information of a bivariate Gaussian with correlation rho, in nats."""
    return -0.5 * np.log(1.0 - rho * rho)
