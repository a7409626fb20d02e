"""Device parallel-tempered sampler (Sec. III) against the oracle's sampler on the same
seeded start ensemble, seed and likelihood.

Positions are bit-exact functions of (seed, start state) while every accept/reject
decision agrees; decisions are float comparisons of lnL differences, so with the
float64 likelihood (|dlnL| ~ 1e-10 here) they agree except with probability ~1e-9
each, and positions and counters are compared exactly.  With the mixed-precision
likelihood (|dlnL| ~ 1e-4) a decision within that distance of its threshold may
flip; the test then requires agreement on all but a few walkers."""
import math

import numpy as np
import pytest

import mbh_inputs as I

pytestmark = pytest.mark.gpu
PROBS = np.array(I.PT_PROBS)


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


def _x_of_theta(th):
    x = np.array(th, dtype=float).copy()
    x[0], x[6], x[8] = math.log(th[0]), math.cos(th[6]), math.sin(th[8])
    return x


@pytest.fixture(scope="module")
def case(oracle, M, WL):
    g = I.grid_month()
    th_raw, snr = I.draw_source(I.rng(0), g["t_obs"])
    z = I.noise_normals(I.rng(0, 100), g["n"])
    src = WL.build_source(g, th_raw, snr, z)
    S = oracle.psd(oracle.freqs(g))
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
    d_o, _ = oracle.make_data(th_o, g, z, S)
    ref_g = M.het_prepare_reference(src.data, src.theta_inj, 64)
    ref_o = oracle.het_prepare(th_o, g, d_o, S, 64)
    lo, hi = I.prior_box(g["t_obs"])
    T, W = 4, 32
    x0 = _x_of_theta(th_o)
    scale = np.abs(x0) * 2e-6 + 1e-5 * (hi - lo) * np.array([0, 0, 1, 1, 0, 1, 1, 1, 1, 1, 0])
    x = I.draw_pt_ensemble(I.rng(63), x0, T, W, scale, lo, hi)
    return dict(g=g, src=src, S=S, d_o=d_o, ref_g=ref_g, ref_o=ref_o, lo=lo, hi=hi, T=T, W=W,
                x=x, x0=x0, scale=scale, betas=I.pt_betas(T, 50.0))


def _gpu_run(M, WL, c, n_iter, precision="fp64", seed=5, graph=True, ref=None):
    pt = M.PTSampler(WL.to_dev(c["x"]), c["betas"], c["lo"], c["hi"], ref=ref or c["ref_g"],
                     walkers=c["W"], probs=PROBS, seed=seed, precision=precision)
    pt.run(n_iter, graph=graph)
    x, out = pt.state()
    cnt, step = pt.counters()
    return pt, x.cpu().numpy(), out.cpu().numpy(), cnt, step


def _oracle_run(oracle, c, n_iter, seed=5):
    out0 = oracle.het_loglike(oracle.pt_theta(c["x"]), c["ref_o"])
    return oracle.pt_run_het(c["x"], out0, c["T"], c["W"], c["betas"], c["lo"], c["hi"], PROBS, 2.0,
                             seed, 0, n_iter, c["ref_o"])


def _lnl_close(a, b, dd, rel=1e-6):
    scale = 0.5 * (dd + np.abs(b[2]) + 2 * np.abs(b[1]))
    assert np.all(np.abs(a[0] - b[0]) <= rel * scale)


@pytest.mark.parametrize("n_iter", [1, 12])
def test_pt_fp64_matches_oracle(M, WL, oracle, case, n_iter):
    _, xg, og, cg, step = _gpu_run(M, WL, case, n_iter)
    xo, oo, co = _oracle_run(oracle, case, n_iter)
    assert step == n_iter
    assert np.array_equal(cg, co), (cg, co)
    assert np.array_equal(xg, xo)
    _lnl_close(og, oo, case["ref_o"]["dd"])
    acc = co[4 * case["T"]:8 * case["T"]].sum()
    assert 0 < acc < co[:4 * case["T"]].sum()          # both branches exercised
    assert co[8 * case["T"] + 1:9 * case["T"]].sum() > 0   # some swaps accepted


@pytest.mark.parametrize("precision", ["mixed", "mixed_f32"])
def test_pt_mixed_matches_oracle(M, WL, oracle, case, precision):
    """Mixed precisions against the oracle's float64 sampler: positions identical but where an
    acceptance test sits within the likelihood's error of its threshold.  "mixed" (fused half
    steps, the extended-precision heterodyne): |dlnL| <= 1e-3 for every walker; "mixed_f32"
    (fused half steps, float32 ratios): hot chains wander far from the reference, where that
    path is held to 1e-6 of the terms, the cold chain stays near it."""
    _, xg, og, cg, _ = _gpu_run(M, WL, case, 3, precision=precision)
    xo, oo, co = _oracle_run(oracle, case, 3)
    same = np.all(xg == xo, axis=0)
    assert same.mean() >= (0.99 if precision == "mixed" else 0.95), same.mean()
    assert np.abs(cg - co).sum() <= 6
    d = np.abs(og[0] - oo[0])
    if precision == "mixed":
        assert d[same].max() <= 1e-3
        return
    scale = 0.5 * (case["ref_o"]["dd"] + np.abs(oo[2]) + 2 * np.abs(oo[1]))
    assert np.all((d / scale)[same] < 1e-6)
    cold = same & (np.arange(d.size) < case["W"])
    assert np.median(d[cold]) < 1e-3


def test_pt_graph_equals_plain_launches(M, WL, case):
    _, x1, o1, c1, _ = _gpu_run(M, WL, case, 5, graph=True)
    _, x2, o2, c2, _ = _gpu_run(M, WL, case, 5, graph=False)
    assert np.array_equal(x1, x2) and np.array_equal(o1, o2) and np.array_equal(c1, c2)


def test_pt_seed_changes_chain(M, WL, case):
    _, x1, _, _, _ = _gpu_run(M, WL, case, 2, seed=5)
    _, x2, _, _, _ = _gpu_run(M, WL, case, 2, seed=6)
    assert not np.array_equal(x1, x2)


def test_pt_best_and_reference_refresh(M, WL, case):
    """Sec. III B refresh: the best cold walker becomes the new reference and every walker is
    rescored against it; the stored lnL equals a plain batch evaluation of the new reference."""
    import torch
    pt, xg, og, _, _ = _gpu_run(M, WL, case, 4, precision="mixed")
    W = case["W"]
    xb, ob = pt.best(0)
    k = int(np.argmax(og[0, :W]))
    assert np.array_equal(xb, xg[:, k]) and ob[0] == og[0, :W].max()
    thb = xb.copy()
    thb[0], thb[6], thb[8] = math.exp(xb[0]), math.acos(xb[6]), math.asin(xb[8])
    ref2 = M.het_prepare_reference(case["src"].data, thb, 64)
    pt.set_ref(ref2)
    x, out = pt.state()
    th = x.clone()
    th[0], th[6], th[8] = torch.exp(x[0]), torch.acos(x[6]), torch.asin(x[8])
    N = x.shape[1]
    plain = M.het_loglike_batch([ref2], [0, N], th, "mixed")
    # theta(x) on the host side of this check uses torch's exp/acos/asin; the lnL of the
    # rescored walkers must agree to the mixed path's accuracy
    assert torch.max(torch.abs(plain[0] - out[0])).item() < 1e-2
    pt.run(2)
    _, step = pt.counters()
    assert step == 6


def test_pt_direct_backend_matches_oracle(M, WL, oracle):
    """Module 1 form: the direct (full-grid) likelihood drives the same sampler."""
    g = I.grid_small(n=2048)
    th_raw, snr = I.draw_source(I.rng(0), g["t_obs"])
    z = I.noise_normals(I.rng(0, 100), g["n"])
    src = WL.build_source(g, th_raw, snr, z)
    S = oracle.psd(oracle.freqs(g))
    th_o = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
    d_o, _ = oracle.make_data(th_o, g, z, S)
    lo, hi = I.prior_box(g["t_obs"])
    T, W = 2, 16
    x0 = _x_of_theta(th_o)
    x = I.draw_pt_ensemble(I.rng(64), x0, T, W, np.abs(x0) * 1e-5 + 1e-4 * (hi - lo) * (x0 == 0),
                           lo, hi)
    betas = I.pt_betas(T)
    pt = M.PTSampler(WL.to_dev(x), betas, lo, hi, data=src.data, walkers=W, probs=PROBS, seed=9,
                     precision="fp64")
    pt.run(3)
    xg, og = (t.cpu().numpy() for t in pt.state())
    cg, _ = pt.counters()
    out0 = oracle.direct(oracle.pt_theta(x), g, d_o, S)
    xo, oo, co = oracle.pt_run_direct(x, out0, T, W, betas, lo, hi, PROBS, 2.0, 9, 0, 3, g, d_o, S)
    assert np.array_equal(cg, co) and np.array_equal(xg, xo)
    dd = oracle.inner(d_o, d_o, S, g["df"])
    _lnl_close(og, oo, dd)


def test_pt_invalid_arguments(M, WL, case):
    c = case
    xd = WL.to_dev(c["x"])
    with pytest.raises(M.MBHError):   # odd walkers
        M.PTSampler(xd[:, :4 * 31].contiguous(), c["betas"], c["lo"], c["hi"], ref=c["ref_g"], walkers=31)
    with pytest.raises(M.MBHError):   # both likelihoods
        M.PTSampler(xd, c["betas"], c["lo"], c["hi"], ref=c["ref_g"], data=c["src"].data, walkers=c["W"])
    with pytest.raises(M.MBHError):   # negative probability
        M.PTSampler(xd, c["betas"], c["lo"], c["hi"], ref=c["ref_g"], walkers=c["W"],
                    probs=(1.1, -0.1, 0, 0))
    with pytest.raises(M.MBHError):   # a <= 1
        M.PTSampler(xd, c["betas"], c["lo"], c["hi"], ref=c["ref_g"], walkers=c["W"], a=1.0)


@pytest.mark.parametrize("W", [1500, 3000, 5000])
def test_pt_large_ensembles_match_oracle(M, WL, oracle, case, W):
    """Ensembles with several walkers per swap-kernel thread (the swap kernel's register
    prefetch of 2, 4 and 8 walkers per thread): one iteration, float64, against the oracle."""
    T = 3
    lo, hi = case["lo"], case["hi"]
    th_o = case["x0"].copy()   # reference at the ensemble's centre
    th_o[0], th_o[6], th_o[8] = math.exp(th_o[0]), math.acos(th_o[6]), math.asin(th_o[8])
    ref_o = oracle.het_prepare(th_o, case["g"], case["d_o"], case["S"], 16)
    ref_g = M.het_prepare_reference(case["src"].data, th_o, 16)
    x = I.draw_pt_ensemble(I.rng(66, W), case["x0"], T, W, case["scale"], lo, hi)
    betas = I.pt_betas(T, 20.0)
    pt = M.PTSampler(WL.to_dev(x), betas, lo, hi, ref=ref_g, walkers=W, probs=PROBS, seed=11,
                     precision="fp64")
    pt.run(1)
    xg, og = (t.cpu().numpy() for t in pt.state())
    cg, _ = pt.counters()
    out0 = oracle.het_loglike(oracle.pt_theta(x), ref_o)
    xo, oo, co = oracle.pt_run_het(x, out0, T, W, betas, lo, hi, PROBS, 2.0, 11, 0, 1, ref_o)
    assert np.array_equal(cg, co)
    assert np.array_equal(xg, xo)
    assert co[8 * T + 1:9 * T].sum() > 0


def test_pt_ladder_adaptation_matches_oracle(M, WL, oracle, case):
    """Ladder adaptation on the device against the oracle: the ladder after 12 iterations to
    float64 rounding (the logarithm and exponential of the two libraries may differ in the
    last bit), positions and counters exactly."""
    c = case
    b0 = np.array([1.0, 0.9, 0.8, 0.0])
    pt = M.PTSampler(WL.to_dev(c["x"]), b0, c["lo"], c["hi"], ref=c["ref_g"], walkers=c["W"],
                     probs=PROBS, seed=5, precision="fp64", adapt=(10.0, 200.0))
    pt.run(12)
    xg, og = (t.cpu().numpy() for t in pt.state())
    cg, _ = pt.counters()
    bg = pt.betas()
    out0 = oracle.het_loglike(oracle.pt_theta(c["x"]), c["ref_o"])
    xo, oo, co, bo = oracle.pt_run_het(c["x"], out0, c["T"], c["W"], b0, c["lo"], c["hi"], PROBS, 2.0,
                                       5, 0, 12, c["ref_o"], adapt=(10.0, 200.0), return_betas=True)
    assert np.array_equal(cg, co) and np.array_equal(xg, xo)
    np.testing.assert_allclose(bg, bo, rtol=1e-13)
    assert not np.allclose(bo, b0) and bo[0] == 1.0 and bo[-1] == 0.0


@pytest.mark.parametrize("precision", ["mixed_f32", "mixed"])
def test_pt_fused_half_steps_equal_separate_launches(M, WL, case, precision):
    """A half step as one fused heterodyne launch (proposal in the walker setup, acceptance in
    the epilogue; the float32-ratio kernel, or the extended kernel for "mixed") against
    proposal, likelihood and acceptance as separate launches.  The likelihood arithmetic is the
    same; the walker constants are compiled into two kernels, so a last-bit difference may flip
    a decision sitting on its threshold."""
    c = case
    runs = []
    for fuse in (True, False):
        pt = M.PTSampler(WL.to_dev(c["x"]), c["betas"], c["lo"], c["hi"], ref=c["ref_g"], walkers=c["W"],
                         probs=PROBS, seed=21, precision=precision, fuse=fuse)
        pt.run(4)
        x, out = (t.cpu().numpy() for t in pt.state())
        cnt, step = pt.counters()
        runs.append((x, out, cnt, step))
    (xa, oa, ca, sa), (xb, ob, cb, sb) = runs
    same = np.all(xa == xb, axis=0)
    assert sa == sb == 4 and same.mean() >= 0.97, same.mean()
    assert np.abs(ca - cb).sum() <= 4
    d = np.abs(oa[0] - ob[0])[same]
    assert d.max() < 1e-6 * np.abs(ob[0][same]).max() + 1e-6


SEED_STEP = 0x9E3779B97F4A7C15


def _ens_refs(M, oracle, c, n):
    """n references around the case's source (the first at the ensemble centre)."""
    th0 = c["x0"].copy()
    th0[0], th0[6], th0[8] = math.exp(th0[0]), math.acos(th0[6]), math.asin(th0[8])
    ths = [th0] + [I.perturb(th0, np.full((11, 1), 10.0 ** (-4 - e)) * (1 - 2 * (e % 2)))[:, 0]
                   for e in range(1, n)]
    refs_g = [M.het_prepare_reference(c["src"].data, th, 32) for th in ths]
    refs_o = [oracle.het_prepare(th, c["g"], c["d_o"], c["S"], 32) for th in ths]
    return refs_g, refs_o


def test_pt_multi_ensemble_matches_oracle(M, WL, oracle, case):
    """Three ensembles, one reference each, stepping together: ensemble e equals the oracle's
    single-ensemble sampler with seed + e 0x9E3779B97F4A7C15 (float64; positions and counters
    exactly)."""
    c = case
    n, T, W = 3, c["T"], c["W"]
    refs_g, refs_o = _ens_refs(M, oracle, c, n)
    xs = [I.draw_pt_ensemble(I.rng(68, e), c["x0"], T, W, c["scale"], c["lo"], c["hi"]) for e in range(n)]
    pt = M.PTSampler(WL.to_dev(np.concatenate(xs, 1)), c["betas"], c["lo"], c["hi"], refs=refs_g,
                     walkers=W, probs=PROBS, seed=7, precision="fp64")
    pt.run(5)
    xg = pt.state()[0].cpu().numpy()
    cg, step = pt.counters()
    assert step == 5
    for e in range(n):
        out0 = oracle.het_loglike(oracle.pt_theta(xs[e]), refs_o[e])
        seed_e = (7 + e * SEED_STEP) % (1 << 64)
        xo, _, co = oracle.pt_run_het(xs[e], out0, T, W, c["betas"], c["lo"], c["hi"], PROBS, 2.0,
                                      seed_e, 0, 5, refs_o[e])
        assert np.array_equal(xg[:, e * T * W:(e + 1) * T * W], xo), e
        assert np.array_equal(cg[e * 10 * T:(e + 1) * 10 * T], co), e
    xb, ob = pt.best(0, ensemble=2)
    og = pt.state()[1].cpu().numpy()[0, 2 * T * W:2 * T * W + W]
    assert ob[0] == og.max()


def test_pt_multi_ensemble_fused_equals_alone(M, WL, oracle, case):
    """Float32-ratio precision, fused half steps: each ensemble of a joint run is bit-identical to the
    same ensemble run alone (its seed, its walkers, its reference)."""
    c = case
    n, T, W = 3, c["T"], c["W"]
    refs_g, _ = _ens_refs(M, oracle, c, n)
    xs = [I.draw_pt_ensemble(I.rng(69, e), c["x0"], T, W, c["scale"], c["lo"], c["hi"]) for e in range(n)]
    pt = M.PTSampler(WL.to_dev(np.concatenate(xs, 1)), c["betas"], c["lo"], c["hi"], refs=refs_g,
                     walkers=W, probs=PROBS, seed=9, precision="mixed_f32")
    pt.run(3)
    xg = pt.state()[0].cpu().numpy()
    cg, _ = pt.counters()
    for e in range(n):
        one = M.PTSampler(WL.to_dev(xs[e]), c["betas"], c["lo"], c["hi"], ref=refs_g[e], walkers=W,
                          probs=PROBS, seed=(9 + e * SEED_STEP) % (1 << 64), precision="mixed_f32")
        one.run(3)
        x1 = one.state()[0].cpu().numpy()
        c1, _ = one.counters()
        assert np.array_equal(xg[:, e * T * W:(e + 1) * T * W], x1), e
        assert np.array_equal(cg[e * 10 * T:(e + 1) * 10 * T], c1), e
