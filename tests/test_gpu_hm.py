"""Higher harmonics (Sec. II A, Eqs. 7-9; stand-in "W0-HM") on the GPU against the oracle:
templates, the direct likelihood, the heterodyne reference (band, edges, summary data) and
likelihood, and the Module-1 sampler with higher-mode templates, all float64.  Tolerances as
in the (2,2) parity tests: templates within 1e-8 of max|h|; lnL within 1e-6 of the size of
the terms; edges bit-exact.  The mixed-precision templates and fused direct likelihood are
held to the (2,2) mixed tolerances; the MBH_MIXED heterodyne to |dlnL| <= 1e-3 absolute against
the oracle, the float32-ratio form to its stated figures."""
import math

import numpy as np
import pytest

import mbh_inputs as I
from edge_rule import f32_edge_count

pytestmark = pytest.mark.gpu
ALL = 0x3F


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


def _hm_case(oracle, M, WL, snr_override=None):
    """Higher-mode injection (q = 0.35, M_T = 5e5) in noise on the 30-day record; each side
    builds its own data from the shared draws."""
    import torch
    g = I.grid_month()
    th_raw, snr = I.draw_source(I.rng(0), g["t_obs"], mt_range=(5e5, 5e5))
    th_raw[I.I_Q] = 0.35
    if snr_override is not None:
        snr = snr_override
    z = I.noise_normals(I.rng(0, 100), g["n"])
    S = oracle.psd(oracle.freqs(g))
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
    d_o = oracle.template_hm(th_o, oracle.freqs(g), g["t_obs"], ALL) + oracle.noise(S, g["df"], z)
    psd = M.mbh_psd_aet(g)
    th_g = th_o.copy()   # the same injection parameters on both sides
    d_g = M.template_batch(g, WL.to_dev(th_g.reshape(11, 1)), "fp64", modes=ALL)[0].contiguous()
    M.mbh_noise_aet(g, torch.from_numpy(np.ascontiguousarray(z)).cuda(), psd, out=d_g, accumulate=True)
    data = M.Data(g, d_g, psd)
    walk = WL.walkers(th_o, 24, 0, lo=1e-5, hi=1e-3)
    return dict(g=g, S=S, th=th_o, d_o=d_o, data=data, walk=walk, snr=snr,
                dd_o=oracle.inner(d_o, d_o, S, g["df"]))


@pytest.fixture(scope="module")
def case(oracle, M, WL):
    return _hm_case(oracle, M, WL)


@pytest.fixture(scope="module")
def loud_case(oracle, M, WL):
    return _hm_case(oracle, M, WL, 1000.0)


def _close(gpu, ora, dd, rel=1e-6):
    scale = 0.5 * (dd + np.abs(ora[2]) + 2 * np.abs(ora[1]))
    err = np.abs(gpu[0] - ora[0])
    assert np.all(err <= rel * scale), (err / scale).max()


@pytest.mark.parametrize("modes", [ALL, 0x2, 0x20, 0x9])
def test_templates(M, WL, oracle, case, modes):
    g, th = case["g"], case["walk"][:, :4]
    h_g = M.template_batch(g, WL.to_dev(th), "fp64", modes=modes).cpu().numpy()
    h_o = oracle.template_batch(th, g, modes)
    assert np.abs(h_o).max() > 0
    assert np.abs(h_g - h_o).max() <= 1e-8 * np.abs(h_o).max()


def test_single_mode_mask_is_w0(M, WL, case):
    g, th = case["g"], WL.to_dev(case["walk"][:, :3])
    a = M.template_batch(g, th, "fp64", modes=1).cpu().numpy()
    b = M.template_batch(g, th, "fp64").cpu().numpy()
    assert np.array_equal(a, b)


def test_direct(M, WL, oracle, case):
    th = case["walk"]
    out_g = M.direct_loglike_batch_hm(case["data"], WL.to_dev(th), ALL).cpu().numpy()
    out_o = oracle.direct(th, case["g"], case["d_o"], case["S"], ALL)
    _close(out_g, out_o, case["dd_o"])
    # the (2,2)-only model fits this data worse than the full one at the injection
    o22 = M.direct_loglike_batch_hm(case["data"], WL.to_dev(case["th"].reshape(11, 1)), 1).cpu().numpy()
    oall = M.direct_loglike_batch_hm(case["data"], WL.to_dev(case["th"].reshape(11, 1)), ALL).cpu().numpy()
    assert o22[0, 0] < oall[0, 0] - 1.0


def test_het_reference_and_likelihood(M, WL, oracle, case):
    ref_g = M.het_prepare_reference(case["data"], case["th"], 64, modes=ALL)
    ref_o = oracle.het_prepare(case["th"], case["g"], case["d_o"], case["S"], 64, ALL)
    assert ref_g.modes == ALL
    rg = ref_g.read()
    assert np.array_equal(rg["edges"], ref_o["edges"])
    np.testing.assert_allclose(rg["summary"], ref_o["summary"], rtol=1e-7,
                               atol=1e-9 * np.abs(ref_o["summary"]).max())
    th = case["walk"]
    out_g = M.het_loglike_batch([ref_g], [0, th.shape[1]], WL.to_dev(th), "fp64").cpu().numpy()
    out_o = oracle.het_loglike(th, ref_o)
    _close(out_g, out_o, case["dd_o"])
    # band of all modes covers the (2,2) band
    _, band22 = oracle.het_edges(case["th"], case["g"], 64)
    assert rg["edges"][0] <= band22[0] and rg["edges"][-1] >= band22[1]


@pytest.mark.parametrize("which", ["case", "loud_case"])
def test_het_mixed_higher_modes(M, WL, oracle, which, request):
    """MBH_MIXED heterodyne of a six-mode reference (per mode group: the phase and time
    differences to the reference at f2 = 2f/m and one transfer, in double-float) against the
    oracle: |dlnL| <= 1e-3 absolute for every walker, 1e-6..1e-4, 1e-4..1e-3 and 1e-3..1e-1
    from the reference, on the SNR-392 source and on the same source at SNR 1000."""
    c = request.getfixturevalue(which)
    ref_g = M.het_prepare_reference(c["data"], c["th"], 64, modes=ALL)
    ref_o = oracle.het_prepare(c["th"], c["g"], c["d_o"], c["S"], 64, ALL)
    for lo, hi in ((1e-6, 1e-4), (1e-4, 1e-3), (1e-3, 1e-1)):
        th = WL.walkers(c["th"], 64, 0, source=7, lo=lo, hi=hi)
        out_m = M.het_loglike_batch([ref_g], [0, th.shape[1]], WL.to_dev(th), "mixed").cpu().numpy()
        out_o = oracle.het_loglike(th, ref_o)
        d = np.abs(out_m[0] - out_o[0])
        print(f"six modes SNR {c['snr']:.0f} {lo:g}..{hi:g}: mixed vs oracle p50/max", np.median(d), d.max())
        assert d.max() <= 1e-3, (lo, hi, d.max())
    # the reference itself: delta = 0 up to rounding
    out_m = M.het_loglike_batch([ref_g], [0, 1], WL.to_dev(c["th"].reshape(11, 1)), "mixed").cpu().numpy()
    out_f = M.het_loglike_batch([ref_g], [0, 1], WL.to_dev(c["th"].reshape(11, 1)), "fp64").cpu().numpy()
    assert abs(out_m[0, 0] - out_f[0, 0]) < 1e-5


@pytest.fixture(scope="module")
def year_case(oracle, M, WL):
    """The benchmark's higher-mode source: workload 2's injection with q = min(q, 0.35) (odd-m
    modes present) at its SNR (122), in noise on the 1-yr grid, 256 bins."""
    import torch
    g = I.grid_year()
    th_raw, snr = WL.injection(2, g, 0)
    th_raw = th_raw.copy()
    th_raw[I.I_Q] = min(th_raw[I.I_Q], 0.35)
    z = I.noise_normals(I.rng(2, 150), g["n"])
    f = oracle.freqs(g)
    S = oracle.psd(f)
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
    d_o = oracle.template_hm(th_o, f, g["t_obs"], ALL) + oracle.noise(S, g["df"], z)
    psd = M.mbh_psd_aet(g)
    d_g = M.template_batch(g, WL.to_dev(th_o.reshape(11, 1)), "fp64", modes=ALL)[0].contiguous()
    M.mbh_noise_aet(g, torch.from_numpy(np.ascontiguousarray(z)).cuda(), psd, out=d_g, accumulate=True)
    data = M.Data(g, d_g, psd)
    ref_g = M.het_prepare_reference(data, th_o, 256, modes=ALL)
    ref_o = oracle.het_prepare(th_o, g, d_o, S, 256, ALL)
    return dict(g=g, th=th_o, ref_g=ref_g, ref_o=ref_o, snr=snr)


def test_het_mixed_higher_modes_float32_edges(M, WL, oracle, year_case):
    """Per-edge precision with six modes: on the benchmark's higher-mode source about half of
    the 257 edges take the float32 ratio of the float32 higher-mode path (the rule recomputed
    from the summary data and the modes' shares of h0), and MBH_MIXED stays within |dlnL| <= 1e-3 of the oracle (32 sampled
    walkers) and of the float64 kernel (every walker), 1e-3..1e-1 and 1e-6..1e-3 from the
    reference."""
    c = year_case
    ref_g, ref_o = c["ref_g"], c["ref_o"]
    np.testing.assert_array_equal(ref_g.read()["edges"], ref_o["edges"])
    # kappa_e: the reference's mode-group shares u_g = h0_g/h0 summed in modulus, per channel
    g = c["g"]
    fe = g["f0"] + ref_o["edges"] * g["df"]
    h0 = oracle.template_hm(c["th"], fe, g["t_obs"], ALL)
    share = np.zeros(h0.shape)
    with np.errstate(all="ignore"):
        for gmask in (0x11, 0x22, 0x04, 0x08):
            hg = oracle.template_hm(c["th"], fe, g["t_obs"], gmask)
            share += np.where(np.abs(h0) > 0, np.abs(hg / h0), 0.0)
    kappa = np.maximum(1.0, share.max(axis=0))
    lo, hi = f32_edge_count(ref_g, g, kappa, rtol=1e-5)   # the library's kappa: from float32 shares
    print(f"six modes, SNR {c['snr']:.0f}: {ref_g.f32_edges} float32-ratio edges of {ref_g.bins + 1} "
          f"(rule: {lo}..{hi})")
    assert lo <= ref_g.f32_edges <= hi and ref_g.f32_edges >= 64
    for lo_p, hi_p, W in ((1e-3, 1e-1, 16384), (1e-6, 1e-3, 4096)):
        th = WL.walkers(c["th"], W, 2, source=9, lo=lo_p, hi=hi_p)
        o64 = M.het_loglike_batch([ref_g], [0, W], WL.to_dev(th), "fp64").cpu().numpy()
        omx = M.het_loglike_batch([ref_g], [0, W], WL.to_dev(th), "mixed").cpu().numpy()
        d = np.abs(omx[0] - o64[0])
        print(f"  {lo_p:g}..{hi_p:g}: mixed vs fp64 p50/p99/max", np.median(d), np.quantile(d, 0.99), d.max())
        assert d.max() <= 1e-3
        sample = np.arange(0, W, W // 32)
        out_o = oracle.het_loglike(np.ascontiguousarray(th[:, sample]), ref_o)
        err = np.abs(omx[0, sample] - out_o[0])
        print("  mixed vs oracle sampled: p50/max", np.median(err), err.max())
        assert err.max() <= 1e-3


def test_het_mixed_f32_higher_modes(M, WL, oracle, case):
    """The float32-ratio form (MBH_MIXED_F32) of the same: near the reference |dlnL| ~ 1e-4, and
    within 1e-6 of the terms for every walker (its error grows with <h|h>)."""
    ref_g = M.het_prepare_reference(case["data"], case["th"], 64, modes=ALL)
    ref_o = oracle.het_prepare(case["th"], case["g"], case["d_o"], case["S"], 64, ALL)
    near = WL.walkers(case["th"], 64, 0, source=7, lo=1e-6, hi=1e-4)
    for th, tol in ((near, 2e-3), (case["walk"], None)):
        out_m = M.het_loglike_batch([ref_g], [0, th.shape[1]], WL.to_dev(th), "mixed_f32").cpu().numpy()
        out_o = oracle.het_loglike(th, ref_o)
        _close(out_m, out_o, case["dd_o"])
        if tol is not None:
            d = np.abs(out_m[0] - out_o[0])
            assert np.median(d) < 1e-3 and d.max() < tol, (np.median(d), d.max())


def test_mixed_batch_of_both_kinds(M, WL, case):
    """A mixed launch holding a (2,2) and a higher-mode source gives each the result it gets
    alone (the plan splits them by kernel)."""
    ref_hm = M.het_prepare_reference(case["data"], case["th"], 32, modes=ALL)
    ref_22 = M.het_prepare_reference(case["data"], case["th"], 32)
    th = case["walk"][:, :10]
    both = np.concatenate([th, th], 1)
    out = M.het_loglike_batch([ref_22, ref_hm], [0, 10, 20], WL.to_dev(both), "mixed").cpu().numpy()
    a = M.het_loglike_batch([ref_22], [0, 10], WL.to_dev(th), "mixed").cpu().numpy()
    b = M.het_loglike_batch([ref_hm], [0, 10], WL.to_dev(th), "mixed").cpu().numpy()
    assert np.array_equal(out[:, :10], a) and np.array_equal(out[:, 10:], b)


def test_mixed_templates_and_direct(M, WL, oracle, case):
    """Mixed-precision higher-mode templates (complex64) and the float32-response fused direct
    likelihood (MBH_MIXED_F32), with the (2,2) float32-response tolerances: templates within
    2e-5 of max|h| per channel, lnL within 1e-5 of the terms; supports bit-exact."""
    g, th = case["g"], case["walk"][:, :4]
    h_g = M.template_batch(g, WL.to_dev(th), "mixed", modes=ALL).cpu().numpy()
    h_o = oracle.template_batch(th, g, ALL)
    for w in range(th.shape[1]):
        for c in range(3):
            ref = np.abs(h_o[w, c]).max()
            assert np.abs(h_g[w, c] - h_o[w, c]).max() <= 2e-5 * ref
    np.testing.assert_array_equal(h_g[:, 0] == 0, h_o[:, 0] == 0)
    out_g = M.direct_loglike_batch_hm(case["data"], WL.to_dev(case["walk"]), ALL, "mixed_f32").cpu().numpy()
    out_o = oracle.direct(case["walk"], g, case["d_o"], case["S"], ALL)
    _close(out_g, out_o, case["dd_o"], rel=1e-5)


@pytest.mark.parametrize("loud", [False, True])
def test_direct_mixed_higher_modes(M, WL, oracle, case, loud_case, loud):
    """The double-float direct likelihood (MBH_MIXED) with the six modes on the 30-day source at
    SNR 392 and 1000: |dlnL| <= 1e-3 absolute against the oracle (24 walkers 1e-5..1e-3), and
    within 1e-6 of the terms of the float64 kernel; mode masks of one and of several groups."""
    c = loud_case if loud else case
    g, th = c["g"], WL.to_dev(c["walk"])
    out_o = oracle.direct(c["walk"], g, c["d_o"], c["S"], ALL)
    out_g = M.direct_loglike_batch_hm(c["data"], th, ALL, "mixed").cpu().numpy()
    err = np.abs(out_g[0] - out_o[0])
    print(f"six-mode direct MBH_MIXED, SNR {c['snr']:.0f}: abs p50/max", np.median(err), err.max())
    assert err.max() <= 1e-3
    for modes in (0x2, 0x9, ALL):
        a = M.direct_loglike_batch_hm(c["data"], th, modes, "mixed").cpu().numpy()
        b = M.direct_loglike_batch_hm(c["data"], th, modes, "fp64").cpu().numpy()
        scale = 0.5 * (c["data"].dd + np.abs(b[2]) + 2 * np.abs(b[1]))
        print(f"  modes 0x{modes:x}: vs float64 abs max", np.abs(a[0] - b[0]).max())
        assert np.all(np.abs(a[0] - b[0]) <= 1e-6 * scale) and np.abs(a[0] - b[0]).max() <= 1e-3


def test_invalid_mode_masks(M, WL, case):
    th = WL.to_dev(case["walk"][:, :2])
    for bad in (0x40, 0x0):
        with pytest.raises(M.MBHError):
            M.template_batch(case["g"], th, "fp64", modes=bad)
        with pytest.raises(M.MBHError):
            M.direct_loglike_batch_hm(case["data"], th, bad)
        with pytest.raises(M.MBHError):
            M.het_prepare_reference(case["data"], case["th"], 16, modes=bad)


def test_sampler_direct_higher_modes(M, WL, oracle):
    """Module-1 sampler with higher-mode templates (the Sec. III C higher-mode posterior is
    sampled this way): positions bit-identical to the oracle's sampler."""
    import torch
    g = I.grid_small(n=1536)
    th_raw, snr = I.draw_source(I.rng(0), g["t_obs"], mt_range=(4e5, 4e5))
    th_raw[I.I_Q] = 0.4
    S = oracle.psd(oracle.freqs(g))
    th = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
    z = I.noise_normals(I.rng(0, 100), g["n"])
    d_o = oracle.template_hm(th, oracle.freqs(g), g["t_obs"], ALL) + oracle.noise(S, g["df"], z)
    psd = M.mbh_psd_aet(g)
    d_g = M.template_batch(g, WL.to_dev(th.reshape(11, 1)), "fp64", modes=ALL)[0].contiguous()
    M.mbh_noise_aet(g, torch.from_numpy(np.ascontiguousarray(z)).cuda(), psd, out=d_g, accumulate=True)
    data = M.Data(g, d_g, psd)
    lo, hi = I.prior_box(g["t_obs"])
    x0 = th.copy()
    x0[0], x0[6], x0[8] = math.log(th[0]), math.cos(th[6]), math.sin(th[8])
    T, W = 2, 8
    x = I.draw_pt_ensemble(I.rng(65), x0, T, W, np.abs(x0) * 1e-5 + 1e-4 * (hi - lo) * (x0 == 0), lo, hi)
    betas = I.pt_betas(T)
    probs = np.array(I.PT_PROBS)
    pt = M.PTSampler(WL.to_dev(x), betas, lo, hi, data=data, walkers=W, probs=probs, seed=3,
                     precision="fp64", modes=ALL)
    pt.run(2)
    xg, og = (t.cpu().numpy() for t in pt.state())
    cg, _ = pt.counters()
    out0 = oracle.direct(oracle.pt_theta(x), g, d_o, S, ALL)
    xo, oo, co = oracle.pt_run_direct(x, out0, T, W, betas, lo, hi, probs, 2.0, 3, 0, 2, g, d_o, S, ALL)
    assert np.array_equal(cg, co) and np.array_equal(xg, xo)
    _close(og, oo, oracle.inner(d_o, d_o, S, g["df"]))
