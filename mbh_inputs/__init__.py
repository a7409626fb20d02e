"""Seeded synthetic inputs for the batched LISA MBHB likelihood workloads.

This module is shared by the oracle tests, the GPU tests and the benchmark.  It
holds none of the method's arithmetic: it only draws source parameters from the
priors (Table I of arXiv:2111.01064, with the narrower ranges of the workloads),
perturbation factors for walker batches, and standard-normal arrays from which
each side builds its own Gaussian noise realisation.  The SNR-setting distance
scale, the waveform, the response, the PSD and the noise scaling are computed by
each side with its own code.

Parameter vector (Sec. II A): theta = [M_T (solar masses, detector frame),
q = m2/m1 in (0, 1], a1, a2, D_L (Gpc), phi_ref, iota, lambda, beta, psi,
t_ref (s)].  Batches are returned as SoA float64 arrays of shape (11, W).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2111_01064
N_PARAMS = 11
(I_MT, I_Q, I_A1, I_A2, I_DL, I_PHI, I_IOTA, I_LAM, I_BETA, I_PSI,
 I_TREF) = range(N_PARAMS)

YEAR_S = 31557600.0   # Julian year; 2,103,840 samples at 15 s
DAY_S = 86400.0


def rng(workload: int, source: int = 0) -> np.random.Generator:
    """PCG64 stream for (workload index, source index)."""
    return np.random.Generator(np.random.PCG64(SEED_BASE + 1000 * workload + source))


# Frequency grids f_k = f0 + k*df, k in [0, n).  t_obs bounds the observation
# window [0, t_obs] in which a template's time-frequency track must lie.
def grid_month() -> dict:
    """30-day record: df = 1/(30 d), 16384 bins starting at bin 260 (~1e-4 Hz)."""
    df = 1.0 / (30.0 * DAY_S)
    return dict(f0=260 * df, df=df, n=16384, t_obs=30.0 * DAY_S)


def grid_year() -> dict:
    """1 yr at 15 s cadence: rfft bins k = 1..1,051,920, df = 1/yr."""
    df = 1.0 / YEAR_S
    return dict(f0=df, df=df, n=1051920, t_obs=YEAR_S)


def grid_small(n: int = 4099, bin0: int = 260, days: float = 30.0) -> dict:
    """A short grid for quick parity cases (same df as the 30-day record)."""
    df = 1.0 / (days * DAY_S)
    return dict(f0=bin0 * df, df=df, n=n, t_obs=days * DAY_S)


def draw_source(g: np.random.Generator, t_obs: float, *, mt_range=(1e5, 1e7),
                qinv_range=(1.0, 10.0), t_margin=(0.3, 0.95)) -> tuple[np.ndarray, float]:
    """One injection: M_T log-uniform, m1/m2 uniform, spins U[-0.99, 0.99],
    isotropic sky and orientation, t_ref inside the window.  D_L is a 1 Gpc
    placeholder; the returned SNR target (log-uniform 100-1000) is met by the
    caller's own distance rescaling."""
    th = np.empty(N_PARAMS)
    th[I_MT] = math.exp(g.uniform(math.log(mt_range[0]), math.log(mt_range[1])))
    th[I_Q] = 1.0 / g.uniform(*qinv_range)
    th[I_A1] = g.uniform(-0.99, 0.99)
    th[I_A2] = g.uniform(-0.99, 0.99)
    th[I_DL] = 1.0
    th[I_PHI] = g.uniform(0.0, 2 * math.pi)
    th[I_IOTA] = math.acos(g.uniform(-1.0, 1.0))
    th[I_LAM] = g.uniform(0.0, 2 * math.pi)
    th[I_BETA] = math.asin(g.uniform(-1.0, 1.0))
    th[I_PSI] = g.uniform(0.0, math.pi)
    th[I_TREF] = g.uniform(t_margin[0] * t_obs, t_margin[1] * t_obs)
    snr = math.exp(g.uniform(math.log(100.0), math.log(1000.0)))
    return th, snr


def draw_prior_batch(g: np.random.Generator, W: int, t_obs: float) -> np.ndarray:
    """W templates from the brute-force search prior (Table I shapes, with the
    mass range 1e5-1e7 and spins within +-0.99): D_L uniform in [1e-2, 1e3] Gpc."""
    th = np.empty((N_PARAMS, W))
    th[I_MT] = np.exp(g.uniform(math.log(1e5), math.log(1e7), W))
    th[I_Q] = 1.0 / g.uniform(1.0, 10.0, W)
    th[I_A1] = g.uniform(-0.99, 0.99, W)
    th[I_A2] = g.uniform(-0.99, 0.99, W)
    th[I_DL] = g.uniform(1e-2, 1e3, W)
    th[I_PHI] = g.uniform(0.0, 2 * math.pi, W)
    th[I_IOTA] = np.arccos(g.uniform(-1.0, 1.0, W))
    th[I_LAM] = g.uniform(0.0, 2 * math.pi, W)
    th[I_BETA] = np.arcsin(g.uniform(-1.0, 1.0, W))
    th[I_PSI] = g.uniform(0.0, math.pi, W)
    th[I_TREF] = g.uniform(0.0, t_obs, W)
    return th


# Scale of the additive perturbation per parameter (relative perturbations are
# used for M_T, q and D_L).  Angles use their prior range; t_ref uses 1000 s
# (about twice the 1 AU light time) and spins their +-0.99 range.
_ADD_SCALE = {I_A1: 1.98, I_A2: 1.98, I_PHI: 2 * math.pi, I_IOTA: math.pi,
              I_LAM: 2 * math.pi, I_BETA: math.pi, I_PSI: math.pi, I_TREF: 1000.0}
_REL = (I_MT, I_Q, I_DL)


def perturbation(g: np.random.Generator, W: int, lo: float = 1e-3, hi: float = 1e-1) -> np.ndarray:
    """Perturbation draws eps of shape (11, W): |eps| log-uniform in [lo, hi],
    random sign.  Apply with `perturb`."""
    mag = np.exp(g.uniform(math.log(lo), math.log(hi), (N_PARAMS, W)))
    sign = np.where(g.uniform(size=(N_PARAMS, W)) < 0.5, -1.0, 1.0)
    return mag * sign


def perturb(theta0: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """Walkers around theta0: relative for M_T, q, D_L; additive (eps x scale)
    for the others.  q is kept in (0, 1], spins in [-0.99, 0.99], and the
    latitude and inclination inside their ranges."""
    W = eps.shape[1]
    th = np.repeat(np.asarray(theta0, dtype=np.float64)[:, None], W, axis=1)
    for i in _REL:
        th[i] = th[i] * (1.0 + eps[i])
    for i, s in _ADD_SCALE.items():
        th[i] = th[i] + eps[i] * s
    th[I_Q] = np.minimum(th[I_Q], 1.0)
    th[I_A1] = np.clip(th[I_A1], -0.99, 0.99)
    th[I_A2] = np.clip(th[I_A2], -0.99, 0.99)
    th[I_IOTA] = np.clip(th[I_IOTA], 1e-3, math.pi - 1e-3)
    th[I_BETA] = np.clip(th[I_BETA], -math.pi / 2 + 1e-3, math.pi / 2 - 1e-3)
    return th


def draw_uneven_batch(g: np.random.Generator, n_sources: int, bins=(64, 512),
                      walkers=(128, 4096)) -> tuple[np.ndarray, np.ndarray]:
    """Per-source bin counts U{bins[0]..bins[1]} and walker counts log-uniform in
    [walkers[0], walkers[1]) (the uneven multi-source batch)."""
    nb = g.integers(bins[0], bins[1] + 1, n_sources)
    nw = np.round(np.exp(g.uniform(math.log(walkers[0]), math.log(walkers[1]), n_sources))).astype(np.int64)
    return nb.astype(np.int64), nw


def draw_requests(g: np.random.Generator, n: int, size=(64, 4096), pool: int = 4096,
                  rate: float = 1.0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Serving requests: sizes log-uniform in [size[0], size[1]], start offsets inside a
    per-source pool of `pool` walkers, and Poisson inter-arrival gaps at `rate` (per s)."""
    sz = np.round(np.exp(g.uniform(math.log(size[0]), math.log(size[1]), n))).astype(np.int64)
    start = (g.uniform(size=n) * (pool - sz + 1)).astype(np.int64)
    gaps = g.exponential(1.0 / rate, n)
    return sz, start, gaps


def noise_normals(g: np.random.Generator, n: int, channels: int = 3) -> np.ndarray:
    """Standard normals of shape (channels, n, 2): real and imaginary parts."""
    return g.standard_normal((channels, n, 2))


def with_distance(theta: np.ndarray, dl_gpc) -> np.ndarray:
    """Copy of theta with D_L replaced (scalar or per-walker)."""
    th = np.array(theta, dtype=np.float64, copy=True)
    th[I_DL] = dl_gpc
    return th


# ---- parallel-tempered sampler inputs (Sec. III) -----------------------------
# The sampler moves x = [ln M_T, q, a1, a2, D_L, phi_ref, cos iota, lambda,
# sin beta, psi, t_ref]; its prior is uniform in x on the box of Table I.
PT_PROBS = (0.85, 0.04, 0.03, 0.08)   # stretch, all 8 sky modes, longitudinal, latitudinal


def prior_box(t_obs: float) -> tuple[np.ndarray, np.ndarray]:
    """Lower and upper bounds of x from Table I (t_ref in [0, t_obs])."""
    lo = np.array([math.log(1e5), 5e-2, -1.0, -1.0, 1e-2, 0.0, -1.0, 0.0, -1.0, 0.0, 0.0])
    hi = np.array([math.log(1e8), 1.0, 1.0, 1.0, 1e3, 2 * math.pi, 1.0, 2 * math.pi, 1.0,
                   math.pi, t_obs])
    return lo, hi


def pt_betas(T: int, t_max: float = 100.0) -> np.ndarray:
    """Inverse temperatures: 1, geometric up to 1/t_max, and 0 (the prior) last."""
    if T == 1:
        return np.ones(1)
    b = np.zeros(T)
    if T > 2:
        b[:T - 1] = t_max ** (-np.arange(T - 1) / (T - 2))
    else:
        b[0] = 1.0
    return b


def draw_pt_ensemble(g: np.random.Generator, x0: np.ndarray, T: int, W: int, scale: np.ndarray,
                     lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """T*W sampler positions (11, T*W) around x0: x0 + scale * N(0, 1), clipped
    into the prior box."""
    x = x0[:, None] + scale[:, None] * g.standard_normal((N_PARAMS, T * W))
    return np.clip(x, lo[:, None], hi[:, None])
