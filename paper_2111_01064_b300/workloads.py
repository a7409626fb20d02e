"""Synthetic workloads built on the GPU through the library only.

The seeded draws (injection parameters, SNR target, walker perturbations,
standard normals) come from ``mbh_inputs``; every step of the method (PSD,
injection template, noise scaling, the SNR used to set D_L) runs in the
library's kernels.  Used by bench.py and the GPU tests.

Workloads (the shapes of the paper's LDC-1A analysis, Sec. II-III; the LDC data
themselves are not available, so these seeded stand-ins are used):
  0  30-day record, 16384 bins from ~1e-4 Hz; one injection (SNR 100-1000) in
     noise; 64 walkers perturbed 1e-3 around it; heterodyne with 128 bins.
  1  1 yr at 15 s: 1,051,920 bins; 4096 prior-drawn templates (direct lnL).
  2  1 yr grid; reference = injection; 8 x 2048 = 16384 walkers perturbed
     1e-3..1e-1 per parameter; 256 bins.
  3  64 sources on 30-day records, bins U{64..512}, walkers log-uniform 128-4096.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

import mbh_inputs as I

from . import mbhlike as M


@dataclasses.dataclass
class Source:
    grid: dict
    psd: torch.Tensor          # (3, n) float64
    d: torch.Tensor            # (3, n) complex128
    data: M.Data
    theta_inj: np.ndarray      # (11,), D_L set for the target SNR
    snr: float


def snr_distance(grid: dict, theta: np.ndarray, snr_target: float, psd: torch.Tensor,
                 zero_data: M.Data | None = None) -> float:
    """D_L (Gpc) giving optimal SNR sqrt(<h|h>) = snr_target (h scales as 1/D_L)."""
    th = np.array(theta, dtype=np.float64).copy()
    th[I.I_DL] = 1.0
    tt = torch.from_numpy(th.reshape(11, 1)).cuda()
    h = M.template_batch(grid, tt, "fp64")
    if zero_data is None:
        zero_data = M.Data(grid, torch.zeros((3, grid["n"]), dtype=torch.complex128, device="cuda"), psd)
    hh = float(M.direct_loglike_stored(zero_data, h, "fp64")[2, 0])
    return float(np.sqrt(hh) / snr_target)


def build_source(grid: dict, theta_raw: np.ndarray, snr_target: float, z: np.ndarray | None) -> Source:
    psd = M.mbh_psd_aet(grid)
    dl = snr_distance(grid, theta_raw, snr_target, psd)
    th = I.with_distance(theta_raw, dl)
    tt = torch.from_numpy(th.reshape(11, 1)).cuda()
    d = M.template_batch(grid, tt, "fp64")[0].contiguous()
    if z is not None:
        M.mbh_noise_aet(grid, torch.from_numpy(np.ascontiguousarray(z)).cuda(), psd, out=d,
                        accumulate=True)
    data = M.Data(grid, d, psd)
    return Source(grid=grid, psd=psd, d=d, data=data, theta_inj=th, snr=snr_target)


def injection(workload: int, grid: dict, source: int = 0):
    g = I.rng(workload, source)
    return I.draw_source(g, grid["t_obs"])


def source_for(workload: int, grid: dict, source: int = 0, noise: bool = True) -> Source:
    th, snr = injection(workload, grid, source)
    z = I.noise_normals(I.rng(workload, 100 + source), grid["n"]) if noise else None
    return build_source(grid, th, snr, z)


def walkers(theta0: np.ndarray, W: int, workload: int, source: int = 0, lo: float = 1e-3,
            hi: float = 1e-1) -> np.ndarray:
    eps = I.perturbation(I.rng(workload, 200 + source), W, lo, hi)
    return np.ascontiguousarray(I.perturb(theta0, eps))


def to_dev(theta: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(theta, dtype=np.float64)).cuda()


@dataclasses.dataclass
class UnevenBatch:
    sources: list
    refs: list
    bins: np.ndarray
    walkers: np.ndarray
    offsets: np.ndarray
    theta: np.ndarray          # (11, W) walkers of all sources, grouped by source


def uneven_batch(n_sources: int = 64, grid: dict | None = None, workload: int = 3,
                 lo: float = 1e-5, hi: float = 1e-3, walkers=(128, 4096)) -> UnevenBatch:
    """Sources with distinct seeds (injection, noise) on the 30-day grid, bins U{64..512},
    walkers log-uniform 128-4096 per source, perturbed lo..hi around each injection."""
    g = grid or I.grid_month()
    nb, nw = I.draw_uneven_batch(I.rng(workload, 999), n_sources, walkers=walkers)
    sources, refs, thetas = [], [], []
    for s in range(n_sources):
        src = source_for(workload, g, source=s)
        sources.append(src)
        refs.append(M.het_prepare_reference(src.data, src.theta_inj, int(nb[s])))
        thetas.append(walkers_for(src.theta_inj, int(nw[s]), workload, s, lo, hi))
    offsets = np.concatenate([[0], np.cumsum(nw)]).astype(np.int64)
    return UnevenBatch(sources=sources, refs=refs, bins=nb, walkers=nw, offsets=offsets,
                       theta=np.ascontiguousarray(np.concatenate(thetas, axis=1)))


def walkers_for(theta0, W, workload, source, lo, hi):
    return walkers(theta0, W, workload, source, lo, hi)
