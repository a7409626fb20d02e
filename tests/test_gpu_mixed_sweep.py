"""MBH_MIXED across randomly drawn sources at the loud end of the workloads' SNR range (1000),
on the 1-yr grid: masses 1e5-1e7, mass ratios 1-10, spins, sky position, orientation and
coalescence time drawn as the workload injections are, in noise.  Every walker of a
4096-walker batch near the reference (1e-6..1e-3) and far from it (1e-3..1e-1) within
|dlnL| <= 1e-3 of the float64 heterodyne kernel (itself held to the oracle in the parity
tests), for the (2,2) mode and for six modes; the double-float direct likelihood of 64
templates near the injection within 1e-3 of the float64 direct kernel.  The per-edge
precision rule (float32-ratio edges within the error budget, the |delta| check, the modes'
cancellation weight) meets sources it was not tuned on."""
import numpy as np
import pytest

import mbh_inputs as I

pytestmark = pytest.mark.gpu
ALL = 0x3F
SNR = 1000.0
W = 4096


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01064_b300 import mbhlike
    mbhlike.lib()
    return mbhlike


@pytest.fixture(scope="module")
def WL(M):
    from paper_2111_01064_b300 import workloads
    return workloads


def _source(M, WL, k, modes):
    """Source k (its own draws) at SNR 1000 in noise; the data carry the template's modes."""
    import torch
    g = I.grid_year()
    th_raw, _ = I.draw_source(I.rng(900 + k), g["t_obs"])
    z = I.noise_normals(I.rng(900 + k, 100), g["n"])
    if modes == 1:
        src = WL.build_source(g, th_raw, SNR, z)
        return src.data, src.theta_inj
    psd = M.mbh_psd_aet(g)
    th = I.with_distance(th_raw, WL.snr_distance(g, th_raw, SNR, psd))
    d = M.template_batch(g, WL.to_dev(th.reshape(11, 1)), "fp64", modes=modes)[0].contiguous()
    M.mbh_noise_aet(g, torch.from_numpy(np.ascontiguousarray(z)).cuda(), psd, out=d, accumulate=True)
    return M.Data(g, d, psd), th


def _het_check(M, WL, data, th0, k, modes):
    ref = M.het_prepare_reference(data, th0, 256, modes=modes)
    worst = []
    for r, (lo, hi) in enumerate(((1e-6, 1e-3), (1e-3, 1e-1))):
        th = WL.to_dev(WL.walkers(th0, W, 9, 2 * k + r, lo=lo, hi=hi))
        o64 = M.het_loglike_batch([ref], [0, W], th, "fp64").cpu().numpy()
        omx = M.het_loglike_batch([ref], [0, W], th, "mixed").cpu().numpy()
        d = np.abs(omx[0] - o64[0])
        worst.append(d.max())
        print(f"source {k} modes 0x{modes:x}: {ref.f32_edges} float32 edges, {lo:g}..{hi:g}: "
              f"abs p50/p99/max {np.median(d):.2e} {np.quantile(d, 0.99):.2e} {d.max():.2e}")
    assert max(worst) <= 1e-3


@pytest.mark.parametrize("k", range(6))
def test_mixed_random_sources(M, WL, k):
    data, th0 = _source(M, WL, k, 1)
    _het_check(M, WL, data, th0, k, 1)
    th = WL.to_dev(WL.walkers(th0, 64, 9, 100 + k, lo=1e-6, hi=1e-3))
    a = M.direct_loglike_batch(data, th, "mixed").cpu().numpy()
    b = M.direct_loglike_batch(data, th, "fp64").cpu().numpy()
    d = np.abs(a[0] - b[0])
    print(f"source {k}: direct abs max {d.max():.2e}")
    assert d.max() <= 1e-3


@pytest.mark.parametrize("k", range(3))
def test_mixed_random_sources_six_modes(M, WL, k):
    data, th0 = _source(M, WL, 10 + k, ALL)
    _het_check(M, WL, data, th0, 10 + k, ALL)
    th = WL.to_dev(WL.walkers(th0, 16, 9, 110 + k, lo=1e-6, hi=1e-3))
    a = M.direct_loglike_batch_hm(data, th, ALL, "mixed").cpu().numpy()
    b = M.direct_loglike_batch_hm(data, th, ALL, "fp64").cpu().numpy()
    d = np.abs(a[0] - b[0])
    print(f"source {10 + k} six modes: direct abs max {d.max():.2e}")
    assert d.max() <= 1e-3
