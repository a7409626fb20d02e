"""GPU (CUDA, through the C ABI) against the FP64 CPU oracle on the same seeded
inputs.  Each side builds its own data from the shared draws (mbh_inputs): its own
PSD, injection template, noise scaling and SNR distance; the tests compare the
results element by element.

Tolerances (floating point):
  * float64 path: |dlnL| <= 1e-6 * scale with scale = (<d|d> + <h|h> + 2|<d|h>|)/2
    (relative 1e-6 is ill-conditioned near lnL ~ 0, so it is taken against the
    size of the terms that cancel); templates within 1e-8 of max|h| (phases of up
    to ~1e7 rad are reproduced to ~1e-9 rad);
  * mixed path ("mixed", MBH_MIXED): heterodyne |dlnL| <= 1e-3 absolute for every walker,
    near the reference and far from it, on sources of SNR 122 to 1000 (the edge values are
    formed relative to the reference in double-float); the direct mixed path (template and
    products in double-float) within 1e-3 absolute on the same sources, near the injection
    and at prior draws;
  * float32-ratio heterodyne ("mixed_f32"): its error grows with <h|h>; held to its stated
    figures at the benchmark's SNR-122 source; the float32-response direct path within 1e-5
    of the terms;
  * integer bookkeeping (band, edges) bit-exact.
"""
import math

import numpy as np
import pytest

import mbh_inputs as I
from edge_rule import f32_edge_count

pytestmark = pytest.mark.gpu


def _lnl_err(gpu, ora, dd):
    scale = 0.5 * (dd + np.abs(ora[2]) + 2 * np.abs(ora[1]))
    return np.abs(gpu[0] - ora[0]), scale


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


@pytest.fixture(scope="module")
def month(oracle, M, WL):
    g = I.grid_month()
    th_raw, snr = I.draw_source(I.rng(0), g["t_obs"])
    z = I.noise_normals(I.rng(0, 100), g["n"])
    src = WL.build_source(g, th_raw, snr, z)
    f = oracle.freqs(g)
    S = oracle.psd(f)
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
    d_o, _ = oracle.make_data(th_o, g, z, S)
    walk_g = WL.walkers(src.theta_inj, 64, 0, lo=1e-4, hi=1e-3)
    walk_o = WL.walkers(th_o, 64, 0, lo=1e-4, hi=1e-3)
    return dict(g=g, src=src, S=S, f=f, th_o=th_o, d_o=d_o, walk_g=walk_g, walk_o=walk_o,
                dd_o=oracle.inner(d_o, d_o, S, g["df"]))


def test_psd(month, M):
    S_g = M.mbh_psd_aet(month["g"]).cpu().numpy()
    np.testing.assert_allclose(S_g, month["S"], rtol=1e-13)


def test_snr_distance(month):
    dg, do = month["src"].theta_inj[I.I_DL], month["th_o"][I.I_DL]
    assert abs(dg / do - 1) < 1e-12


def test_data_dd(month):
    assert month["src"].data.dd == pytest.approx(month["dd_o"], rel=1e-12)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 2e-5)])
def test_template(month, M, WL, oracle, prec, tol):
    g = month["g"]
    th = month["walk_o"][:, :6]
    h_g = M.template_batch(g, WL.to_dev(th), prec).cpu().numpy()
    h_o = oracle.template_batch(th, g)
    for w in range(th.shape[1]):
        for c in range(3):
            ref = np.abs(h_o[w, c]).max()
            err = np.abs(h_g[w, c] - h_o[w, c]).max()
            assert err <= tol * ref, (prec, w, c, err / ref)
    # support bookkeeping is bit-exact
    np.testing.assert_array_equal(h_g[:, 0] == 0, h_o[:, 0] == 0)


def _crossing(oracle, th, t_obs, target, a, b):
    """f in [a, b] with t(f) = target (the oracle's time-frequency map), by bisection."""
    ta = oracle.w0(th, np.array([a]), t_obs)[2][0] - target
    for _ in range(200):
        m = 0.5 * (a + b)
        tm = oracle.w0(th, np.array([m]), t_obs)[2][0] - target
        if (tm < 0) == (ta < 0):
            a, ta = m, tm
        else:
            b = m
    return 0.5 * (a + b)


@pytest.mark.parametrize("bound", ["t=0", "t=t_obs"])
def test_mixed_support_at_time_bounds(month, M, WL, oracle, bound):
    """The support t(f) in [0, t_obs] (Sec. II A, the time-frequency map) decided by the
    mixed templates point by point as by the oracle, on a grid of ~0.5 s steps in t across
    each bound: the mixed chain forms t - t_ref in float32 and falls back to the double-float
    t where the float32 value's rounding bound straddles a bound (here on most points)."""
    g0 = month["g"]
    th = month["th_o"].copy()
    info = oracle.w0_info(th)
    if bound == "t=0":
        fs = _crossing(oracle, th, g0["t_obs"], 0.0, 1e-7, info["fmax"])
    else:   # t_ref just past t_obs: t(f) crosses t_obs below f_max
        th[I.I_TREF] = g0["t_obs"] + 20.0
        fs = _crossing(oracle, th, g0["t_obs"], g0["t_obs"], 0.5 * info["fmax"], info["fmax"])
    h = 1e-7 * fs
    t2 = oracle.w0(th, np.array([fs - h, fs + h]), g0["t_obs"])[2]
    slope = abs(t2[1] - t2[0]) / (2 * h)
    step = 0.5 / slope
    g = dict(f0=fs - 128.5 * step, df=step, n=257, t_obs=g0["t_obs"])
    f = oracle.freqs(g)
    h_o = oracle.template(th, f, g["t_obs"])
    h_m = M.template_batch(g, WL.to_dev(th.reshape(11, 1)), "mixed").cpu().numpy()[0]
    inside = h_o[0] != 0
    assert 50 < inside.sum() < 207   # the bound lies inside the grid
    np.testing.assert_array_equal(h_m[0] != 0, inside)


def test_template_ragged_and_empty(month, M, WL, oracle):
    g = I.grid_small(n=1000 + 37)
    th = month["walk_o"][:, :3]
    h_g = M.template_batch(g, WL.to_dev(th), "fp64").cpu().numpy()
    h_o = oracle.template_batch(th, g)
    np.testing.assert_allclose(h_g, h_o, rtol=0, atol=1e-8 * np.abs(h_o).max())
    e = M.template_batch(g, WL.to_dev(np.zeros((11, 0))), "fp64")
    assert e.shape == (0, 3, g["n"])


def test_direct_fp64(month, M, WL, oracle):
    g, src = month["g"], month["src"]
    out_g = M.direct_loglike_batch(src.data, WL.to_dev(month["walk_g"]), "fp64").cpu().numpy()
    out_o = oracle.direct(month["walk_o"], g, month["d_o"], month["S"])
    err, scale = _lnl_err(out_g, out_o, month["dd_o"])
    print("direct fp64 max rel", (err / scale).max(), "abs", err.max())
    assert np.all(err <= 1e-6 * scale)
    np.testing.assert_allclose(out_g[2], out_o[2], rtol=1e-9)


def test_direct_stored_matches_fused(month, M, WL):
    src = month["src"]
    th = WL.to_dev(month["walk_g"][:, :13])   # ragged against the 4-template tile
    h = M.template_batch(month["g"], th, "fp64")
    a = M.direct_loglike_stored(src.data, h, "fp64").cpu().numpy()
    b = M.direct_loglike_batch(src.data, th, "fp64").cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-9)
    h32 = M.template_batch(month["g"], th, "mixed")
    c = M.direct_loglike_stored(src.data, h32, "mixed").cpu().numpy()
    scale = 0.5 * (src.data.dd + np.abs(b[2]) + 2 * np.abs(b[1]))
    print("stored fp32 vs fp64 max rel", (np.abs(c[0] - b[0]) / scale).max())
    assert np.all(np.abs(c[0] - b[0]) <= 1e-5 * scale)


@pytest.mark.parametrize("prec", ["mixed", "mixed_f32"])
def test_direct_mixed(month, M, WL, oracle, prec):
    g, src = month["g"], month["src"]
    out_g = M.direct_loglike_batch(src.data, WL.to_dev(month["walk_g"]), prec).cpu().numpy()
    out_o = oracle.direct(month["walk_o"], g, month["d_o"], month["S"])
    err, scale = _lnl_err(out_g, out_o, month["dd_o"])
    print(f"direct {prec} max rel", (err / scale).max(), "abs p50/max", np.median(err), err.max())
    assert np.all(err <= 1e-5 * scale)
    if prec == "mixed":
        assert err.max() <= 1e-3


@pytest.fixture(scope="module")
def refs(month, M, oracle):
    g = month["g"]
    ref_g = M.het_prepare_reference(month["src"].data, month["src"].theta_inj, 128)
    ref_o = oracle.het_prepare(month["th_o"], g, month["d_o"], month["S"], 128)
    return ref_g, ref_o


def test_het_prepare(refs):
    ref_g, ref_o = refs
    r = ref_g.read()
    assert r["E"] == ref_o["E"]
    np.testing.assert_array_equal(r["edges"], ref_o["edges"])
    for m in range(6):
        x, y = r["summary"][:, :, m], ref_o["summary"][:, :, m]
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-9 * np.abs(y).max())
    np.testing.assert_allclose(r["h0e"], ref_o["h0e"], rtol=0, atol=1e-8 * np.abs(ref_o["h0e"]).max())
    assert r["dd"] == pytest.approx(ref_o["dd"], rel=1e-12)


def test_het_fp64(month, refs, M, WL, oracle):
    ref_g, ref_o = refs
    W = month["walk_g"].shape[1]
    out_g = M.het_loglike_batch([ref_g], [0, W], WL.to_dev(month["walk_g"]), "fp64").cpu().numpy()
    out_o = oracle.het_loglike(month["walk_o"], ref_o)
    err, scale = _lnl_err(out_g, out_o, ref_o["dd"])
    print("het fp64 max rel", (err / scale).max(), "abs max", err.max())
    assert np.all(err <= 1e-6 * scale)


def test_het_mixed(month, refs, M, WL, oracle):
    ref_g, ref_o = refs
    th_g = WL.walkers(month["src"].theta_inj, 64, 0, lo=1e-6, hi=1e-4)
    th_o = WL.walkers(month["th_o"], 64, 0, lo=1e-6, hi=1e-4)
    out_g = M.het_loglike_batch([ref_g], [0, 64], WL.to_dev(th_g), "mixed").cpu().numpy()
    out_o = oracle.het_loglike(th_o, ref_o)
    err, scale = _lnl_err(out_g, out_o, ref_o["dd"])
    print("het mixed near: abs p50/p99/max", np.median(err), np.quantile(err, 0.99), err.max())
    assert err.max() <= 1e-3
    for lo, hi in ((1e-4, 1e-3), (1e-3, 1e-1)):
        far_g = WL.walkers(month["src"].theta_inj, 256, 0, lo=lo, hi=hi)
        far_o = WL.walkers(month["th_o"], 256, 0, lo=lo, hi=hi)
        far = M.het_loglike_batch([ref_g], [0, 256], WL.to_dev(far_g), "mixed").cpu().numpy()
        ora = oracle.het_loglike(far_o, ref_o)
        err, scale = _lnl_err(far, ora, ref_o["dd"])
        print(f"het mixed {lo:g}..{hi:g}: abs p50/max", np.median(err), err.max())
        assert err.max() <= 1e-3


def test_het_exact_at_reference(month, refs, M, WL):
    ref_g, _ = refs
    th = WL.to_dev(month["src"].theta_inj.reshape(11, 1))
    het = M.het_loglike_batch([ref_g], [0, 1], th, "fp64").cpu().numpy()
    dr = M.direct_loglike_batch(month["src"].data, th, "fp64").cpu().numpy()
    scale = 0.5 * (month["src"].data.dd + abs(dr[2, 0]) + 2 * abs(dr[1, 0]))
    assert abs(het[0, 0] - dr[0, 0]) <= 1e-11 * scale
    mix = M.het_loglike_batch([ref_g], [0, 1], th, "mixed").cpu().numpy()
    assert abs(mix[0, 0] - dr[0, 0]) <= 1e-6
    f32 = M.het_loglike_batch([ref_g], [0, 1], th, "mixed_f32").cpu().numpy()
    assert abs(f32[0, 0] - dr[0, 0]) <= 1e-3


def test_het_multi_source_equals_single(month, M, WL):
    """Walkers of several sources in one launch give the same results as one
    launch per source (deterministic per-walker reduction)."""
    g = month["g"]
    srcs, refs, ths = [], [], []
    for s, nb in enumerate((128, 7, 300)):
        src = WL.source_for(3, g, source=s)
        srcs.append(src)
        refs.append(M.het_prepare_reference(src.data, src.theta_inj, nb))
        ths.append(WL.walkers(src.theta_inj, (33, 1, 70)[s], 3, s, 1e-5, 1e-3))
    off = np.concatenate([[0], np.cumsum([t.shape[1] for t in ths])])
    th = WL.to_dev(np.concatenate(ths, axis=1))
    for prec in ("fp64", "mixed", "mixed_f32"):
        allg = M.het_loglike_batch(refs, off, th, prec).cpu().numpy()
        for s in range(3):
            one = M.het_loglike_batch([refs[s]], [0, ths[s].shape[1]], WL.to_dev(ths[s]), prec).cpu().numpy()
            np.testing.assert_array_equal(allg[:, off[s]:off[s + 1]], one)


def test_het_edge_cases(month, M, WL, oracle):
    src = month["src"]
    r1 = M.het_prepare_reference(src.data, src.theta_inj, 1)
    assert r1.bins == 1
    out = M.het_loglike_batch([r1], [0, 0], WL.to_dev(np.zeros((11, 0))), "mixed")
    assert out.shape == (3, 0)
    # a walker whose support misses most edges (10x the mass): finite, matches the oracle
    far = src.theta_inj.copy()
    far[I.I_MT] *= 10
    ref_o = oracle.het_prepare(month["th_o"], month["g"], month["d_o"], month["S"], 1)
    far_o = month["th_o"].copy()
    far_o[I.I_MT] *= 10
    a = M.het_loglike_batch([r1], [0, 1], WL.to_dev(far.reshape(11, 1)), "fp64").cpu().numpy()
    b = oracle.het_loglike(far_o, ref_o)
    assert np.all(np.isfinite(a))
    assert abs(a[0, 0] - b[0, 0]) <= 1e-6 * (ref_o["dd"] + abs(b[2, 0]) + 2 * abs(b[1, 0]))


def test_invalid_arguments(month, M, WL):
    src = month["src"]
    with pytest.raises(M.MBHError) as e:
        M.het_prepare_reference(src.data, src.theta_inj, 0)
    assert e.value.status == 1
    with pytest.raises(M.MBHError):
        M.mbh_psd_aet(dict(f0=-1.0, df=1e-6, n=10, t_obs=1e6))
    ref = M.het_prepare_reference(src.data, src.theta_inj, 16)
    th = WL.to_dev(month["walk_g"][:, :4])
    with pytest.raises(M.MBHError):
        M.het_loglike_batch([ref, ref], [0, 3, 2], th, "fp64")   # decreasing offsets
    with pytest.raises(M.MBHError):
        M.het_loglike_batch([ref], [0, 4], th, "half")


# ---- full-size cases, sampled against the oracle ---------------------------------------
@pytest.fixture(scope="module")
def year(oracle, M, WL):
    g = I.grid_year()
    th_raw, snr = I.draw_source(I.rng(1), g["t_obs"])
    z = I.noise_normals(I.rng(1, 100), g["n"])
    src = WL.build_source(g, th_raw, snr, z)
    f = oracle.freqs(g)
    S = oracle.psd(f)
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
    d_o, _ = oracle.make_data(th_o, g, z, S)
    return dict(g=g, src=src, S=S, th_o=th_o, d_o=d_o)


def test_direct_full_size_sampled(year, M, WL, oracle):
    """4096 prior-drawn templates on the 1-yr grid (the brute-force search batch),
    in the launch configuration of the benchmark; 3 sampled templates against the
    oracle, the rest through the fp64-vs-mixed agreement."""
    g = year["g"]
    th = I.draw_prior_batch(I.rng(1, 300), 4096, g["t_obs"])
    # put a few templates near the injection so that lnL is not just -<d|d>/2
    th[:, :8] = WL.walkers(year["src"].theta_inj, 8, 1, lo=1e-6, hi=1e-5)
    out64 = M.direct_loglike_batch(year["src"].data, WL.to_dev(th), "fp64").cpu().numpy()
    outm = M.direct_loglike_batch(year["src"].data, WL.to_dev(th), "mixed").cpu().numpy()
    outf = M.direct_loglike_batch(year["src"].data, WL.to_dev(th), "mixed_f32").cpu().numpy()
    sample = [0, 3, 1234]
    tho = th[:, sample].copy()
    tho[:, :2] = WL.walkers(year["th_o"], 8, 1, lo=1e-6, hi=1e-5)[:, [0, 3]]
    out_o = oracle.direct(tho, g, year["d_o"], year["S"])
    err, scale = _lnl_err(out64[:, sample], out_o, year["src"].data.dd)
    print("year direct fp64 sampled rel", err / scale)
    assert np.all(err <= 1e-6 * scale)
    scale_all = 0.5 * (year["src"].data.dd + np.abs(out64[2]) + 2 * np.abs(out64[1]))
    # the double-float template carries the ~1e6-rad phase to ~|Phi| 2^-48, so the error of a
    # template is a fixed fraction (~1e-11) of <h|h>: <= 1e-3 up to SNR ~1000 (<h|h> <= 1e6);
    # the prior also draws nearby heavy binaries with <h|h> up to ~1e9
    d = np.abs(outm[0] - out64[0])
    loud = out64[2] > 1e6
    print("year direct mixed vs fp64 abs p50/max", np.median(d), d[~loud].max(),
          f"({loud.sum()} templates above SNR 1000: max", (d / scale_all)[loud].max(), "of the terms)")
    assert d[~loud].max() <= 1e-3
    assert np.all(d <= 1e-10 * scale_all)
    rel = np.abs(outf[0] - out64[0]) / scale_all
    print("year direct mixed_f32 vs fp64 rel max", rel.max(), "abs max", np.abs(outf[0] - out64[0]).max())
    assert np.all(rel <= 1e-5)
    err, _ = _lnl_err(outm[:, sample], out_o, year["src"].data.dd)
    print("year direct mixed sampled vs oracle abs", err)
    assert err.max() <= 1e-3


def test_direct_mixed_snr1000(M, WL, oracle):
    """The 1-yr source of the heterodyne benchmark made louder (SNR 1000): the double-float
    direct path within |dlnL| <= 1e-3 of the float64 kernel for 256 templates near the
    injection (1e-6..1e-3) and for the 256 prior draws up to SNR 1000, and of the oracle for 3
    sampled ones."""
    g = I.grid_year()
    th_raw, _ = WL.injection(2, g)
    z = I.noise_normals(I.rng(2, 100), g["n"])
    src = WL.build_source(g, th_raw, 1000.0, z)
    th = np.concatenate([WL.walkers(src.theta_inj, 256, 2, lo=1e-6, hi=1e-3),
                         I.draw_prior_batch(I.rng(1, 301), 256, g["t_obs"])], axis=1)
    o64 = M.direct_loglike_batch(src.data, WL.to_dev(th), "fp64").cpu().numpy()
    omx = M.direct_loglike_batch(src.data, WL.to_dev(th), "mixed").cpu().numpy()
    d = np.abs(omx[0] - o64[0])
    quiet = o64[2] <= 1e6   # templates up to SNR 1000 (the rest: a fixed fraction of <h|h>)
    print("SNR 1000 direct mixed vs fp64: near p50/max", np.median(d[:256]), d[:256].max(),
          "prior p50/max (SNR <= 1000)", np.median(d[256:]), d[256:][quiet[256:]].max())
    assert d[:256].max() <= 1e-3 and d[quiet].max() <= 1e-3
    scale = 0.5 * (src.data.dd + np.abs(o64[2]) + 2 * np.abs(o64[1]))
    assert np.all(d <= 1e-10 * scale)
    S = oracle.psd(oracle.freqs(g))
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, 1000.0, S))
    d_o, _ = oracle.make_data(th_o, g, z, S)
    sample = [0, 100, 300]
    tho = th[:, sample].copy()
    tho[:, :2] = WL.walkers(th_o, 256, 2, lo=1e-6, hi=1e-3)[:, sample[:2]]
    out_o = oracle.direct(tho, g, d_o, S)
    err = np.abs(omx[0, sample] - out_o[0])
    print("SNR 1000 direct mixed sampled vs oracle", err)
    assert err.max() <= 1e-3


def test_het_full_size_sampled(year, M, WL, oracle):
    """16384 walkers (8 temperatures x 2048) perturbed 1e-3..1e-1, 256 bins on the
    1-yr grid; 32 sampled walkers against the oracle."""
    g = year["g"]
    ref_g = M.het_prepare_reference(year["src"].data, year["src"].theta_inj, 256)
    ref_o = oracle.het_prepare(year["th_o"], g, year["d_o"], year["S"], 256)
    r = ref_g.read()
    np.testing.assert_array_equal(r["edges"], ref_o["edges"])
    W = 16384
    th_g = WL.walkers(year["src"].theta_inj, W, 2)
    th_o = WL.walkers(year["th_o"], W, 2)
    o64 = M.het_loglike_batch([ref_g], [0, W], WL.to_dev(th_g), "fp64").cpu().numpy()
    omx = M.het_loglike_batch([ref_g], [0, W], WL.to_dev(th_g), "mixed").cpu().numpy()
    sample = np.arange(0, W, W // 32)
    out_o = oracle.het_loglike(np.ascontiguousarray(th_o[:, sample]), ref_o)
    err, scale = _lnl_err(o64[:, sample], out_o, ref_o["dd"])
    assert np.all(err <= 1e-6 * scale)
    err, scale = _lnl_err(omx[:, sample], out_o, ref_o["dd"])
    print("year het mixed sampled: abs p50/max", np.median(err), err.max())
    assert err.max() <= 1e-3
    # every walker, mixed against the float64 kernel (itself held to the oracle above)
    err, _ = _lnl_err(omx, o64, year["src"].data.dd)
    print("year het mixed vs fp64 (SNR 473): abs p50/p99/max", np.median(err), np.quantile(err, 0.99), err.max())
    assert err.max() <= 1e-3


def test_het_mixed_benchmark_accuracy(M, WL):
    """The benchmark's heterodyne batch (workload 2: 16384 walkers 1e-3..1e-1 from the
    injection, 256 bins, 1-yr grid, SNR 122): mixed precision within |dlnL| <= 1e-3 of the
    float64 kernel for every walker; the float32-ratio path for at least 99.5 % of them, none
    beyond 5e-3."""
    g = I.grid_year()
    src = WL.source_for(2, g)
    ref = M.het_prepare_reference(src.data, src.theta_inj, 256)
    W = 16384
    th = WL.to_dev(WL.walkers(src.theta_inj, W, 2))
    o64 = M.het_loglike_batch([ref], [0, W], th, "fp64").cpu().numpy()
    omx = M.het_loglike_batch([ref], [0, W], th, "mixed").cpu().numpy()
    d = np.abs(omx[0] - o64[0])
    print("workload 2 mixed vs fp64: p50/p99/max", np.median(d), np.quantile(d, 0.99), d.max())
    assert d.max() <= 1e-3
    o32 = M.het_loglike_batch([ref], [0, W], th, "mixed_f32").cpu().numpy()
    d = np.abs(o32[0] - o64[0])
    print("workload 2 mixed_f32 vs fp64: p50/p99/max", np.median(d), np.quantile(d, 0.99), d.max(),
          "frac <= 1e-3", np.mean(d <= 1e-3))
    assert np.mean(d <= 1e-3) >= 0.995 and d.max() <= 5e-3


def test_f32_edge_choice(M, WL):
    """The reference's float32-ratio edges follow the per-edge precision rule (recomputed on
    the host from the summary data): on the benchmark's source (SNR 122) and on the same
    source at SNR 1000, where fewer edges qualify."""
    g = I.grid_year()
    th_raw, snr = WL.injection(2, g)
    z = I.noise_normals(I.rng(2, 100), g["n"])
    counts = []
    for target in (snr, 1000.0):
        src = WL.build_source(g, th_raw, target, z)
        ref = M.het_prepare_reference(src.data, src.theta_inj, 256)
        lo, hi = f32_edge_count(ref, g)
        print(f"SNR {target:.0f}: {ref.f32_edges} float32-ratio edges of {ref.bins + 1} (rule: {lo}..{hi})")
        assert lo <= ref.f32_edges <= hi
        counts.append(ref.f32_edges)
    assert counts[0] > counts[1] > 0


@pytest.mark.parametrize("lo,hi,W", [(1e-3, 1e-1, 16384), (1e-6, 1e-3, 4096)])
def test_het_mixed_snr1000(M, WL, oracle, lo, hi, W):
    """Workload 2's source made louder, SNR 1000 (the top of the workloads' SNR range), 256
    bins on the 1-yr grid: every walker within |dlnL| <= 1e-3 of the float64 kernel, and 32
    sampled walkers within 1e-3 of the oracle, far from the reference and near it."""
    g = I.grid_year()
    th_raw, _ = WL.injection(2, g)
    z = I.noise_normals(I.rng(2, 100), g["n"])
    src = WL.build_source(g, th_raw, 1000.0, z)
    ref = M.het_prepare_reference(src.data, src.theta_inj, 256)
    th = WL.walkers(src.theta_inj, W, 2, lo=lo, hi=hi)
    o64 = M.het_loglike_batch([ref], [0, W], WL.to_dev(th), "fp64").cpu().numpy()
    omx = M.het_loglike_batch([ref], [0, W], WL.to_dev(th), "mixed").cpu().numpy()
    d = np.abs(omx[0] - o64[0])
    print(f"SNR 1000 {lo:g}..{hi:g} mixed vs fp64: p50/p99/max", np.median(d), np.quantile(d, 0.99), d.max())
    assert d.max() <= 1e-3
    S = oracle.psd(oracle.freqs(g))
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, 1000.0, S))
    d_o, _ = oracle.make_data(th_o, g, z, S)
    ref_o = oracle.het_prepare(th_o, g, d_o, S, 256)
    np.testing.assert_array_equal(ref.read()["edges"], ref_o["edges"])
    sample = np.arange(0, W, W // 32)
    wo = WL.walkers(th_o, W, 2, lo=lo, hi=hi)
    out_o = oracle.het_loglike(np.ascontiguousarray(wo[:, sample]), ref_o)
    err = np.abs(omx[0, sample] - out_o[0])
    print("SNR 1000 mixed vs oracle sampled: p50/max", np.median(err), err.max())
    assert err.max() <= 1e-3
