"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only makes data: the coupled processes that stand in for the paper's simulations
and MEG recordings, the random trial permutations that define surrogate data sets, and the
bookkeeping of which (series, analysis time point, surrogate) estimates a workload contains.
It holds none of the estimator's arithmetic (no embedding, no distances, no counts, no digamma).

Shapes follow the paper's problem statement: a series is trials x samples (``[R][T]``,
row-major float32), the same layout for source X and target Y (Eq. 3 / Eq. 4 notation:
repetition r, time t).  Surrogates pair target trial r with source trial ``perms[s][r]``; this
is the trial shuffling of Fig. 3 expressed on the source side (TE depends only on the pairing).

All generators draw from ``numpy.random.default_rng(seed)`` (PCG64), run the recursions in
float64, drop ``burn`` leading samples per trial and store float32, so that every consumer
reads identical bits within one run.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

BASE_SEED = 20140728  # publication year/month/day of the paper; seed = BASE_SEED + config id
BURN_IN = 200

# AR(2) pair used by the stationary / non-stationary / surrogate workloads:
#   x_t = AX1 x_{t-1} + AX2 x_{t-2} + eta_x
#   y_t = AY1 y_{t-1} + AY2 y_{t-2} + c(t) x_{t-U_AR} + eta_y
AR_AX = (0.5, -0.2)
AR_AY = (0.4, -0.2)
AR_COUPLING = 0.5
AR_U = 5
AR_SIGMA = 1.0


@dataclass
class Series:
    """One source/target pair: trials x samples arrays plus its embedding parameters."""
    src: np.ndarray            # float32 [R][T]
    tgt: np.ndarray            # float32 [R][T]
    d: int                     # embedding dimension (d_X = d_Y = d)
    tau: int                   # embedding delay
    u: int                     # assumed interaction delay
    perms: Optional[np.ndarray] = None  # int32 [S][R]: surrogate s pairs tgt trial r with src trial perms[s][r]

    @property
    def R(self) -> int:
        return int(self.src.shape[0])

    @property
    def T(self) -> int:
        return int(self.src.shape[1])

    @property
    def S(self) -> int:
        return 0 if self.perms is None else int(self.perms.shape[0])


@dataclass
class Instance:
    """One estimate: a series, an analysis window [t_start, t_start+window) and a pairing."""
    series: int
    t_start: int
    window: int
    perm: int = -1             # -1: original pairing; s >= 0: surrogate s of that series


@dataclass
class Workload:
    name: str
    series: List[Series]
    instances: List[Instance]
    k: int = 4
    # For surrogate-test workloads: per series the analysis start points, the window and S.
    t_starts: Optional[List[List[int]]] = None
    window: Optional[int] = None
    S: int = 0
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def n_points(self, inst: Instance) -> int:
        return self.series[inst.series].R * inst.window

    def joint_dim(self, inst: Instance) -> int:
        return 1 + 2 * self.series[inst.series].d

    def pair_evals(self) -> int:
        """Ordered (i, j != i) point pairs summed over all instances: the work of ONE pass."""
        tot = 0
        for inst in self.instances:
            n = self.n_points(inst)
            tot += n * (n - 1)
        return tot

    def lane_ops(self) -> int:
        """Algorithmic FP32 operations of ONE pass: D subtractions + D abs-max per ordered pair."""
        tot = 0
        for inst in self.instances:
            n = self.n_points(inst)
            tot += n * (n - 1) * 2 * self.joint_dim(inst)
        return tot


# ----------------------------------------------------------------------------------------
# process generators
# ----------------------------------------------------------------------------------------

def ar2_pair(rng: np.random.Generator, R: int, T: int, coupling_start: Optional[int] = 0,
             coupling: float = AR_COUPLING, burn: int = BURN_IN):
    """Unidirectionally coupled AR(2) pair X -> Y with delay AR_U and unit Gaussian noise.

    ``coupling_start``: kept-sample index from which the coupling is on (None: never on).
    """
    L = T + burn
    ex = rng.standard_normal((R, L)) * AR_SIGMA
    ey = rng.standard_normal((R, L)) * AR_SIGMA
    x = np.zeros((R, L))
    y = np.zeros((R, L))
    for t in range(L):
        xt = ex[:, t].copy()
        yt = ey[:, t].copy()
        if t >= 1:
            xt += AR_AX[0] * x[:, t - 1]
            yt += AR_AY[0] * y[:, t - 1]
        if t >= 2:
            xt += AR_AX[1] * x[:, t - 2]
            yt += AR_AY[1] * y[:, t - 2]
        kept = t - burn
        if coupling_start is not None and kept >= coupling_start and t >= AR_U:
            yt += coupling * x[:, t - AR_U]
        x[:, t] = xt
        y[:, t] = yt
    return (np.ascontiguousarray(x[:, burn:], dtype=np.float32),
            np.ascontiguousarray(y[:, burn:], dtype=np.float32))


def pink_noise(rng: np.random.Generator, R: int, L: int) -> np.ndarray:
    """1/f noise per trial by spectral shaping of white Gaussian noise, unit variance."""
    w = rng.standard_normal((R, L))
    f = np.fft.rfft(w, axis=1)
    freqs = np.arange(f.shape[1], dtype=np.float64)
    scale = np.zeros_like(freqs)
    scale[1:] = 1.0 / np.sqrt(freqs[1:])
    p = np.fft.irfft(f * scale[None, :], n=L, axis=1)
    p -= p.mean(axis=1, keepdims=True)
    p /= p.std(axis=1, keepdims=True)
    return p


def pink_pair(rng: np.random.Generator, R: int, T: int, u: int, coupling: float = 0.5,
              burn: int = BURN_IN):
    """MEG-like pair: y = pink_y + coupling * x(t-u), x pink, both unit variance before mixing."""
    L = T + burn
    x = pink_noise(rng, R, L)
    yp = pink_noise(rng, R, L)
    y = yp.copy()
    y[:, u:] += coupling * x[:, :-u]
    return (np.ascontiguousarray(x[:, burn:], dtype=np.float32),
            np.ascontiguousarray(y[:, burn:], dtype=np.float32))


def logistic_ar_pair(rng: np.random.Generator, R: int, T: int, u: int = 5, r_log: float = 3.9,
                     a_y: float = 0.4, coupling: float = 0.5, burn: int = BURN_IN):
    """Logistic-map source (r = 3.9, x0 ~ U(0.1, 0.9)) driving a noisy AR(1) target
    through a squared (nonlinear) coupling: y_t = a_y y_{t-1} + coupling * x_{t-u}^2 + eta."""
    L = T + burn
    x = np.zeros((R, L))
    x[:, 0] = rng.uniform(0.1, 0.9, size=R)
    for t in range(1, L):
        x[:, t] = r_log * x[:, t - 1] * (1.0 - x[:, t - 1])
    ey = rng.standard_normal((R, L))
    y = np.zeros((R, L))
    for t in range(L):
        yt = ey[:, t].copy()
        if t >= 1:
            yt += a_y * y[:, t - 1]
        if t >= u:
            yt += coupling * x[:, t - u] ** 2
        y[:, t] = yt
    return (np.ascontiguousarray(x[:, burn:], dtype=np.float32),
            np.ascontiguousarray(y[:, burn:], dtype=np.float32))


def gaussian_pair_iid(rng: np.random.Generator, R: int, T: int, rho: float):
    """i.i.d. bivariate Gaussian samples (correlation rho) laid out as trials x samples;
    used for the mutual-information special case of the estimator."""
    z1 = rng.standard_normal((R, T))
    z2 = rng.standard_normal((R, T))
    x = z1
    y = rho * z1 + np.sqrt(1.0 - rho * rho) * z2
    return x.astype(np.float32), y.astype(np.float32)


# Table 1: parameters of the three coupled AR(1) scenarios (Eq. 12 - Eq. 16); delays in samples
# (1 kHz sampling, so samples = ms), t counted from the first kept sample of a trial.
AR1_SCENARIOS = {
    "unidirectional": dict(ax=0.75, ay=0.35, byx=0.0, bxy=-0.35, dyx=0, dxy=10),
    "two-step": dict(ax=0.75, ay=0.35, byx=0.0, bxy=-0.35, dyx=0, dxy=10),
    "bidirectional": dict(ax=0.475, ay=0.35, byx=-0.4, bxy=-0.35, dyx=20, dxy=10),
}


def ar1_couplings(name: str, t: np.ndarray):
    """gamma_XY(t), gamma_YX(t) of Eq. 14 - Eq. 16 (tanh ramps, slope 0.05, scaled to 0..1)."""
    p = AR1_SCENARIOS[name]
    ramp = lambda t0: 0.5 * (1.0 + np.tanh(0.05 * (t - t0)))
    if name == "two-step":
        gxy = p["bxy"] * 0.5 * (ramp(1000.0) + ramp(2000.0))
    else:
        gxy = p["bxy"] * ramp(1000.0)
    gyx = p["byx"] * ramp(2000.0)
    return gxy, gyx


def ar1_scenario(rng: np.random.Generator, name: str, R: int = 50, T: int = 3000, burn: int = BURN_IN):
    """Coupled AR(1) pair of Eq. 12 / Eq. 13 with the Table 1 parameters of scenario `name`:
    x(t) = a_X x(t-1) + gamma_YX(t) y(t - d_YX) + eta_X,  y(t) = a_Y y(t-1) + gamma_XY(t) x(t - d_XY) + eta_Y,
    unit-variance Gaussian noise; returns (src = x, tgt = y)."""
    p = AR1_SCENARIOS[name]
    L = T + burn
    ex = rng.standard_normal((R, L))
    ey = rng.standard_normal((R, L))
    gxy, gyx = ar1_couplings(name, np.arange(L, dtype=np.float64) - burn)
    x = np.zeros((R, L))
    y = np.zeros((R, L))
    for t in range(L):
        xt = ex[:, t].copy()
        yt = ey[:, t].copy()
        if t >= 1:
            xt += p["ax"] * x[:, t - 1]
            yt += p["ay"] * y[:, t - 1]
        if p["byx"] != 0.0 and t >= p["dyx"]:
            xt += gyx[t] * y[:, t - p["dyx"]]
        if t >= p["dxy"]:
            yt += gxy[t] * x[:, t - p["dxy"]]
        x[:, t] = xt
        y[:, t] = yt
    return (np.ascontiguousarray(x[:, burn:], dtype=np.float32),
            np.ascontiguousarray(y[:, burn:], dtype=np.float32))


def permutations(rng: np.random.Generator, S: int, R: int) -> np.ndarray:
    """S uniform random permutations of 0..R-1 (surrogate trial pairings), int32 [S][R]."""
    out = np.empty((S, R), dtype=np.int32)
    for s in range(S):
        out[s] = rng.permutation(R).astype(np.int32)
    return out


# ----------------------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------------------

def _surrogate_instances(n_series_t: Sequence[Sequence[int]], window: int, S: int) -> List[Instance]:
    insts = []
    for si, ts in enumerate(n_series_t):
        for t in ts:
            insts.append(Instance(si, t, window, -1))
            for s in range(S):
                insts.append(Instance(si, t, window, s))
    return insts


def config(cid: int, *, n_t: Optional[int] = None, S: Optional[int] = None,
           R: Optional[int] = None, n_pairs: Optional[int] = None) -> Workload:
    """The five benchmark workloads.  Keyword overrides shrink a workload (fewer time points,
    surrogates, trials or channel pairs) for tests; the defaults are the full sizes."""
    rng = np.random.default_rng(BASE_SEED + cid)
    if cid == 1:
        # AR(2) X->Y, 200 trials x 300 samples, d=2, tau=1, u=5, one window of 5 samples
        Rr = R or 200
        src, tgt = ar2_pair(rng, Rr, 300, coupling_start=0)
        s = Series(src, tgt, d=2, tau=1, u=AR_U)
        return Workload("C1 stationary AR(2), 1000 points x 5-D, 1 estimate", [s],
                        [Instance(0, 100, 5, -1)], k=4)
    if cid == 2:
        # coupling switched on at sample 500; 100 analysis points, window 3, d=3, tau=2
        Rr = R or 500
        src, tgt = ar2_pair(rng, Rr, 1000, coupling_start=500)
        s = Series(src, tgt, d=3, tau=2, u=AR_U)
        nt = n_t or 100
        ts = [9 + 9 * j for j in range(nt)]
        return Workload("C2 non-stationary AR(2), 1500 points x 7-D, 100 time points", [s],
                        [Instance(0, t, 3, -1) for t in ts], k=4, t_starts=[ts], window=3)
    if cid == 3:
        # surrogate test: 400 trials, d=3, tau=1, window 3, 50 time points x (1 + 1000)
        Rr = R or 400
        src, tgt = ar2_pair(rng, Rr, 1000, coupling_start=0)
        SS = 1000 if S is None else S
        perms = permutations(rng, SS, Rr)
        s = Series(src, tgt, d=3, tau=1, u=AR_U, perms=perms)
        nt = n_t or 50
        ts = [9 + 18 * j for j in range(nt)]
        return Workload("C3 surrogate test, 1200 points x 7-D, 50 t x (1+1000)", [s],
                        _surrogate_instances([ts], 3, SS), k=4, t_starts=[ts], window=3, S=SS)
    if cid == 4:
        # 20 pink-noise channel pairs with uneven trials / dims / windows, 30 time points each
        npairs = n_pairs or 20
        series, insts = [], []
        nt = n_t or 30
        for p in range(npairs):
            Rp = int(rng.integers(50, 2001)) if R is None else R
            dp = int(rng.integers(1, 6))
            Wp = int(rng.integers(1, 6))
            up = int(rng.integers(2, 21))
            src, tgt = pink_pair(rng, Rp, 600, up)
            series.append(Series(src, tgt, d=dp, tau=1, u=up))
            for j in range(nt):
                insts.append(Instance(p, 24 + 18 * j, Wp, -1))
        return Workload("C4 uneven MEG-like batch, 20 pairs x 30 t, N 50..10000, D 3..11",
                        series, insts, k=4)
    if cid == 5:
        # 4000 trials, d=5, window 3 -> 12000 points x 11-D; 200 t x (1 + 200)
        Rr = R or 4000
        src, tgt = logistic_ar_pair(rng, Rr, 400, u=5)
        SS = 200 if S is None else S
        perms = permutations(rng, SS, Rr)
        s = Series(src, tgt, d=5, tau=1, u=5, perms=perms)
        nt = n_t or 200
        ts = [9 + j for j in range(nt)]
        return Workload("C5 large ensemble, 12000 points x 11-D, 200 t x (1+200)", [s],
                        _surrogate_instances([ts], 3, SS), k=4, t_starts=[ts], window=3, S=SS)
    raise ValueError(f"unknown config {cid}")


def ar1_analysis(name: str = "unidirectional", S: int = 500, R: int = 50, window: int = 300,
                 n_windows: int = None, seed: int = 0) -> Workload:
    """The paper's AR(1) analysis: 50 trials x 3000 samples, d = 1, tau = 1, analysis windows of
    300 samples from sample 200 on (4 windows for the unidirectional scenario, 8 otherwise),
    delays scanned over 1..20 (1..30 for the bidirectional scenario), S surrogates, k = 4.
    The instances hold the original and surrogates at the true delay; a delay scan supplies u."""
    rng = np.random.default_rng(BASE_SEED + 60 + seed + list(AR1_SCENARIOS).index(name))
    src, tgt = ar1_scenario(rng, name, R=R)
    perms = permutations(rng, S, R)
    s = Series(src, tgt, d=1, tau=1, u=AR1_SCENARIOS[name]["dxy"], perms=perms)
    nw = n_windows or (4 if name == "unidirectional" else 8)
    ts = [200 + window * j for j in range(nw)]
    u_hi = 30 if name == "bidirectional" else 20
    return Workload(f"AR(1) {name} scenario (Table 1), {R} trials, windows of {window}", [s],
                    _surrogate_instances([ts], window, S), k=4, t_starts=[ts], window=window, S=S,
                    extra=dict(u_lo=1, u_hi=u_hi))


# ---------------------------------------------------------------------------------------
# Two unidirectionally coupled Lorenz systems X -> Y (Eq. 11): for system i in {X, Y}
#   dU_i/dt = sigma (V_i - U_i)
#   dV_i/dt = U_i (rho_i - W_i) - V_i + gamma_XY(t) V_X(t - delta)^2   (the last term for i = Y only)
#   dW_i/dt = U_i V_i - beta W_i
# The paper analyses the V coordinates and states gamma_XY = 0.3, delta = 45 ms, 1 kHz sampling,
# but not sigma, rho, beta, the solver's time scale or the initial states: those below are this
# implementation's choices (classic Lorenz constants; one sample = 0.02 model time units, so the
# coupling delay is 0.9 units = 45 samples and the autocorrelation of V falls to 1/e within about
# 8 samples; random initial states relaxed for 1000 samples).
LORENZ_SIGMA = 10.0
LORENZ_BETA = 8.0 / 3.0
LORENZ_RHO = (28.0, 28.0)      # rho_X, rho_Y
LORENZ_DT = 0.02               # model time units per sample
LORENZ_SUBSTEPS = 4            # fourth-order Runge-Kutta steps per sample
LORENZ_DELAY = 45              # delta_XY in samples
LORENZ_GAMMA = 0.3
LORENZ_BURN = 1000


def lorenz_pair(rng: np.random.Generator, R: int, T: int, gamma: float = LORENZ_GAMMA,
                delay: int = LORENZ_DELAY, coupled=(1000, 2000), burn: int = LORENZ_BURN,
                substeps: int = LORENZ_SUBSTEPS, dt: float = None):
    """R repetitions of T samples of the Eq. 11 pair; returns (src = V_X, tgt = V_Y) float32.

    ``coupled``: kept-sample interval [a, b) in which gamma_XY = gamma (None: all samples,
    burn-in included); gamma_XY = 0 elsewhere.  The delay-differential equation is integrated
    with classical RK4 on a grid of ``substeps`` steps per sample; the delayed V_X at a step's
    midpoint is the mean of the two neighbouring grid values (linear interpolation), and before
    the first ``delay`` samples the history is the initial state (a constant initial function).
    """
    h = (dt or LORENZ_DT) / substeps
    lag = delay * substeps                      # delay in grid steps
    rho = np.array(LORENZ_RHO).reshape(2, 1)
    u = rng.uniform(-15.0, 15.0, (2, R))
    v = rng.uniform(-15.0, 15.0, (2, R))
    w = rng.uniform(5.0, 40.0, (2, R))
    hist = np.repeat(v[0][None, :], lag + 1, axis=0)   # V_X on the last lag + 1 grid points
    out = np.empty((2, R, T), dtype=np.float32)

    def f(u, v, w, c):
        du = LORENZ_SIGMA * (v - u)
        dv = u * (rho - w) - v
        dv[1] += c
        dw = u * v - LORENZ_BETA * w
        return du, dv, dw

    n_steps = (burn + T) * substeps
    for n in range(n_steps):
        sample = n // substeps - burn               # kept-sample index of this step
        if n % substeps == 0 and sample >= 0:
            out[:, :, sample] = v
        hist[n % (lag + 1)] = v[0]
        on = (coupled is None) or (coupled[0] <= sample < coupled[1])
        g = gamma if on else 0.0
        if g != 0.0:
            x0 = hist[(n + 1) % (lag + 1)]          # V_X(t_n - delta)
            x1 = hist[(n + 2) % (lag + 1)] if lag >= 1 else v[0]   # V_X(t_n + h - delta)
            c0, ch, c1 = g * x0 * x0, g * (0.5 * (x0 + x1)) ** 2, g * x1 * x1
        else:
            c0 = ch = c1 = 0.0
        k1 = f(u, v, w, c0)
        k2 = f(u + 0.5 * h * k1[0], v + 0.5 * h * k1[1], w + 0.5 * h * k1[2], ch)
        k3 = f(u + 0.5 * h * k2[0], v + 0.5 * h * k2[1], w + 0.5 * h * k2[2], ch)
        k4 = f(u + h * k3[0], v + h * k3[1], w + h * k3[2], c1)
        u = u + h / 6.0 * (k1[0] + 2.0 * k2[0] + 2.0 * k3[0] + k4[0])
        v = v + h / 6.0 * (k1[1] + 2.0 * k2[1] + 2.0 * k3[1] + k4[1])
        w = w + h / 6.0 * (k1[2] + 2.0 * k2[2] + 2.0 * k3[2] + k4[2])
    return np.ascontiguousarray(out[0]), np.ascontiguousarray(out[1])


# Embedding of the Lorenz V coordinates for the analyses (the paper uses "optimal" parameters
# without stating them): d = 4 and tau = 3 samples, about half the autocorrelation time. The
# paper's benchmark chunk has 17 = 1 + 2 * 8 joint coordinates, so d = 8 there.
LORENZ_D = 4
LORENZ_TAU = 3


def lorenz_analysis(S: int = 500, R: int = 150, T: int = 3000, d: int = LORENZ_D, tau: int = LORENZ_TAU,
                    seed: int = 0, dt: float = None) -> Workload:
    """The paper's non-stationary Lorenz analysis (Fig. 6): 150 repetitions x 3000 samples, coupling
    gamma_XY = 0.3 with delay 45 samples during samples 1000..2000 only, analysis windows
    200..450, 1600..1850 and 2750..3000 (250 samples), delays scanned over 35..55, S surrogates,
    k = 4.  The instances hold the original and surrogates at the true delay; a delay scan
    supplies u."""
    rng = np.random.default_rng(BASE_SEED + 80 + seed)
    src, tgt = lorenz_pair(rng, R, T, dt=dt)
    perms = permutations(rng, S, R)
    s = Series(src, tgt, d=d, tau=tau, u=LORENZ_DELAY, perms=perms)
    ts = [t for t in (200, 1600, 2750) if t + 250 <= T]
    return Workload(f"Lorenz X->Y (Eq. 11), {R} repetitions, windows of 250", [s],
                    _surrogate_instances([ts], 250, S), k=4, t_starts=[ts], window=250, S=S,
                    extra=dict(u_lo=35, u_hi=55))


def lorenz_robustness(S: int = 100, R: int = 300, d: int = LORENZ_D, tau: int = LORENZ_TAU,
                      trials=(3, 10, 25, 50, 150), seed: int = 0, dt: float = None):
    """The robustness analysis (Fig. 8): coupled Lorenz systems (gamma_XY = 0.3 throughout, delay
    45 samples), repetitions of 300 samples, delays scanned over 30..60.  The paper takes the
    first M = 500 .. 30000 embedded points; here a point set is the first R_M whole repetitions
    over the window 100..299 (200 points each): M = 600, 2000, 5000, 10000, 30000.
    Returns {M: Workload} (one series per M, the first R_M repetitions, S surrogates each)."""
    rng = np.random.default_rng(BASE_SEED + 90 + seed)
    src, tgt = lorenz_pair(rng, R, 300, coupled=None, dt=dt)
    out = {}
    for r_m in trials:
        perms = permutations(rng, S, r_m)
        s = Series(np.ascontiguousarray(src[:r_m]), np.ascontiguousarray(tgt[:r_m]), d=d, tau=tau,
                   u=LORENZ_DELAY, perms=perms)
        out[r_m * 200] = Workload(f"Lorenz robustness, M = {r_m * 200} points", [s],
                                  _surrogate_instances([[100]], 200, S), k=4, t_starts=[[100]],
                                  window=200, S=S, extra=dict(u_lo=30, u_hi=60))
    return out


def paper_chunk(chunks: int = 16, seed: int = 0) -> Workload:
    """The benchmark chunk of the paper's performance test: 30094 points in the 17-D joint space
    (d = 8) of coupled Lorenz data, k = 4.  Here 82 repetitions x a window of 367 samples
    (t' = 133..499, u = 45, tau = 1); ``chunks`` estimates of that shape (the original pairing
    and chunks - 1 trial-shuffled surrogates: same shape and cost, different point sets)."""
    rng = np.random.default_rng(BASE_SEED + 95 + seed)
    src, tgt = lorenz_pair(rng, 82, 500, coupled=None)
    perms = permutations(rng, max(1, chunks - 1), 82)
    s = Series(src, tgt, d=8, tau=1, u=LORENZ_DELAY, perms=perms)
    insts = [Instance(0, 133, 367, -1)] + [Instance(0, 133, 367, c) for c in range(chunks - 1)]
    return Workload("paper benchmark chunk: 30094 points x 17-D (d = 8), Lorenz", [s], insts, k=4)


def sample_instances(w: Workload, n: int, seed: int = 0) -> List[int]:
    """Indices of a seeded, cost-stratified subset of a workload's instances."""
    rng = np.random.default_rng(BASE_SEED + 1000 + seed)
    idx = np.arange(len(w.instances))
    if n >= len(idx):
        return list(idx)
    cost = np.array([w.n_points(i) ** 2 * w.joint_dim(i) for i in w.instances], dtype=np.float64)
    order = idx[np.argsort(cost, kind="stable")]
    strata = np.array_split(order, n)
    return sorted(int(rng.choice(s)) for s in strata if len(s))
