"""Pins of the oracle's parallel-tempered ensemble sampler (Sec. III, the
paragraph after Table I): the Philox4x32-10 generator against its published
known answers, the distribution of the random choices, the sky-mode maps, and
the stationary distributions the sampler must reach on closed-form targets."""
import json
import math
import os

import numpy as np
import pytest

import mbh_inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PROBS = np.array(I.PT_PROBS)


def test_philox_known_answers(oracle):
    kat = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(h, 16) for h in v["ctr"]]
        key = [int(h, 16) for h in v["key"]]
        out = oracle.philox(ctr, key)[0]
        assert [f"{int(o):08x}" for o in out] == v["out"]


def test_choice_statistics(oracle):
    """Kinds with the Sec. III frequencies; complement uniform on the other half;
    z with density ~ 1/sqrt(z) on [1/a, a]; sky modes uniform."""
    W, n, a = 64, 20000, 2.0
    ch = [oracle.pt_choice(7, 3, i % 2, i // 2, W, PROBS, a) for i in range(n)]
    kinds = np.bincount([c["kind"] for c in ch], minlength=4) / n
    assert np.all(np.abs(kinds - PROBS) < 4 * np.sqrt(PROBS * (1 - PROBS) / n) + 1e-9)
    for half in (0, 1):
        js = np.array([c["j"] for i, c in enumerate(ch) if i % 2 == half])
        assert js.min() >= (1 - half) * W // 2 and js.max() < (2 - half) * W // 2
        cnt = np.bincount(js - (1 - half) * W // 2, minlength=W // 2)
        e = len(js) / (W // 2)
        assert ((cnt - e) ** 2 / e).sum() < W // 2 + 6 * math.sqrt(W)   # chi^2, 31 dof
    z = np.sort([c["z"] for c in ch])
    assert z.min() >= 1 / a and z.max() <= a
    cdf = (np.sqrt(a * z) - 1) / (a - 1)
    ks = np.max(np.abs(cdf - (np.arange(1, n + 1) - 0.5) / n))
    assert ks < 1.63 / math.sqrt(n)                                      # KS at 1 %
    sky_all = [c for c in ch if c["kind"] == 1]
    nm = np.bincount([c["n"] * 2 + c["m"] for c in sky_all], minlength=8)
    assert nm.min() > 0.6 * len(sky_all) / 8
    lon = [c for c in ch if c["kind"] == 2]
    assert {c["n"] for c in lon} == {1, 2, 3} and all(c["m"] == 0 for c in lon)
    assert all(c["n"] == 0 and c["m"] == 1 for c in ch if c["kind"] == 3)


def test_sky_maps(oracle):
    """Longitudinal quarter turns move lambda and psi together (mod 2 pi, mod pi);
    the latitudinal mode flips sin beta, cos iota and cos psi; both are group
    actions, so each map has its inverse among the proposals."""
    x = np.array([12.0, 0.5, 0.1, 0.2, 10.0, 1.0, 0.3, 5.9, -0.4, 2.8, 1e5])
    for n in range(4):
        y = oracle.pt_sky(x, n, 0)
        assert y[7] == pytest.approx((x[7] + n * math.pi / 2) % (2 * math.pi), abs=1e-12)
        assert y[9] == pytest.approx((x[9] + n * math.pi / 2) % math.pi, abs=1e-12)
        assert np.array_equal(np.delete(y, [7, 9]), np.delete(x, [7, 9]))
        back = oracle.pt_sky(y, (4 - n) % 4, 0)
        assert back[7] == pytest.approx(x[7], abs=1e-12) and back[9] == pytest.approx(x[9], abs=1e-12)
    y = oracle.pt_sky(x, 0, 1)
    assert (y[8], y[6]) == (-x[8], -x[6])
    assert math.cos(y[9]) == pytest.approx(-math.cos(x[9]), abs=1e-15)
    assert np.array_equal(oracle.pt_sky(y, 0, 1), x)


def _gauss_setup():
    lo, hi = I.prior_box(1e6)
    mu = np.array([math.log(1e6), 0.5, 0.1, 0.0, 500.0, 0.0, 0.0, math.pi, 0.0, 0.0, 5e5])
    sig = np.array([0.3, 0.06, 0.1, 0.0, 50.0, 0.0, 0.15, 0.4, 0.15, 0.0, 5e4])
    return lo, hi, mu, sig


def test_stationary_distribution_tempered(oracle):
    """On a diagonal Gaussian target the chain at inverse temperature beta samples
    N(mu, sigma^2/beta) (truncation negligible on this machine), and the beta = 0
    chain the uniform prior box; a wrong sign, a missing z^(d-1) factor or a wrong
    swap rule shifts these moments far beyond the tolerances."""
    lo, hi, mu, sig = _gauss_setup()
    T, W = 3, 64
    betas = np.array([1.0, 0.25, 0.0])
    g = I.rng(60)
    x = lo[:, None] + (hi - lo)[:, None] * g.random((11, T * W))
    out = oracle.pt_gauss_loglike(x, mu, sig)
    x, out, cnt, tr = oracle.pt_run_gauss(x, out, T, W, betas, lo, hi, PROBS, 2.0, 11, 0, 6000,
                                          mu, sig, trace=True)
    s = tr[1200:].reshape(-1, 11, T, W)
    for t, b in enumerate(betas):
        samp = s[:, :, t, :].transpose(1, 0, 2).reshape(11, -1)
        m, v = samp.mean(1), samp.var(1)
        for p in range(11):
            if sig[p] > 0 and b > 0:
                sd = sig[p] / math.sqrt(b)
                assert abs(m[p] - mu[p]) < 0.15 * sd, (t, p, m[p], mu[p])
                assert abs(v[p] / sd ** 2 - 1) < 0.15, (t, p, v[p], sd ** 2)
            elif b == 0 or sig[p] == 0:
                w = hi[p] - lo[p]
                assert abs(m[p] - 0.5 * (lo[p] + hi[p])) < 0.08 * w, (t, p)
                assert abs(v[p] / (w * w / 12) - 1) < 0.15, (t, p, v[p])
    # bookkeeping: every walker proposes once per iteration; W swap proposals per level
    props = cnt[:4 * T].reshape(T, 4).sum(1)
    assert np.all(props == 6000 * W)
    assert np.all(cnt[9 * T + 1:10 * T] == 6000 * W) and cnt[9 * T] == 0
    assert np.all(cnt[4 * T:8 * T] <= cnt[:4 * T])
    # the stored lnL is that of the stored state
    assert np.array_equal(out, oracle.pt_gauss_loglike(x, mu, sig))


def test_sky_hops_detailed_balance(oracle):
    """With sky-mode hops only, a walker moves on the 8 images of its start; in
    equilibrium it occupies image i with probability ~ exp(lnL_i)."""
    lo, hi = I.prior_box(1e6)
    mu = np.array([0, 0, 0, 0, 0, 0, 0.1, 1.0, 0.2, 1.0, 0], dtype=float)
    sig = np.array([0, 0, 0, 0, 0, 0, 0.6, 1.0, 0.5, 0.8, 0], dtype=float)
    x0 = np.array([14.0, 0.5, 0.0, 0.0, 10.0, 1.0, 0.2, 1.2, 0.3, 0.9, 1e5])
    imgs = np.stack([oracle.pt_sky(x0, n, m) for n in range(4) for m in range(2)], 1)
    p = np.exp(oracle.pt_gauss_loglike(imgs, mu, sig)[0])
    p /= p.sum()
    W = 64
    x = np.repeat(x0[:, None], W, 1)
    out = oracle.pt_gauss_loglike(x, mu, sig)
    probs = np.array([0.0, 0.4, 0.3, 0.3])
    _, _, _, tr = oracle.pt_run_gauss(x, out, 1, W, np.ones(1), lo, hi, probs, 2.0, 5, 0, 4000,
                                      mu, sig, trace=True)
    lam, sb = tr[100:, 7, :].ravel(), tr[100:, 8, :].ravel()
    n = np.round(((lam - x0[7]) / (math.pi / 2))) % 4
    m = (sb < 0).astype(int)
    freq = np.bincount((n * 2 + m).astype(int), minlength=8) / n.size
    assert np.max(np.abs(freq - p)) < 0.02, (freq, p)


def test_het_sampler_bookkeeping(oracle):
    """With the heterodyned likelihood: the stored (lnL, <d|h>, <h|h>) of every
    walker is the oracle's value at its stored position, after moves and swaps."""
    g = I.grid_small(n=2048)
    th, snr = I.draw_source(I.rng(0), g["t_obs"])
    f = oracle.freqs(g)
    S = oracle.psd(f)
    th[I.I_DL] = oracle.snr_distance(th, g, snr, S)
    d, _ = oracle.make_data(th, g, I.noise_normals(I.rng(0, 100), g["n"]), S)
    ref = oracle.het_prepare(th, g, d, S, 32)
    lo, hi = I.prior_box(g["t_obs"])
    x0 = th.copy()
    x0[0], x0[6], x0[8] = math.log(th[0]), math.cos(th[6]), math.sin(th[8])
    T, W = 2, 8
    scale = 1e-4 * (hi - lo)
    x = I.draw_pt_ensemble(I.rng(61), x0, T, W, scale, lo, hi)
    out = oracle.het_loglike(oracle.pt_theta(x), ref)
    x1, out1, cnt = oracle.pt_run_het(x, out, T, W, I.pt_betas(T), lo, hi, PROBS, 2.0, 3, 0, 3, ref)
    assert np.array_equal(out1, oracle.het_loglike(oracle.pt_theta(x1), ref))
    assert cnt[:4 * T].sum() == 3 * T * W and cnt[4 * T:8 * T].sum() > 0
    assert not np.array_equal(x1, x)


def test_direct_sampler_bookkeeping(oracle):
    """Module 1 form (direct likelihood): stored values match the state."""
    g = I.grid_small(n=1024)
    th, snr = I.draw_source(I.rng(0), g["t_obs"])
    f = oracle.freqs(g)
    S = oracle.psd(f)
    th[I.I_DL] = oracle.snr_distance(th, g, snr, S)
    d, _ = oracle.make_data(th, g, I.noise_normals(I.rng(0, 100), g["n"]), S)
    lo, hi = I.prior_box(g["t_obs"])
    x0 = th.copy()
    x0[0], x0[6], x0[8] = math.log(th[0]), math.cos(th[6]), math.sin(th[8])
    T, W = 2, 8
    x = I.draw_pt_ensemble(I.rng(62), x0, T, W, 1e-4 * (hi - lo), lo, hi)
    out = oracle.direct(oracle.pt_theta(x), g, d, S)
    x1, out1, cnt = oracle.pt_run_direct(x, out, T, W, I.pt_betas(T), lo, hi, PROBS, 2.0, 4, 0, 2,
                                         g, d, S)
    assert np.array_equal(out1, oracle.direct(oracle.pt_theta(x1), g, d, S))
    assert cnt[:4 * T].sum() == 2 * T * W


def test_ladder_adaptation_equalises_swap_rates(oracle):
    """Vousden et al. adaptation: from a poor ladder (three temperatures crowded near 1 and the
    prior last) the swap acceptance rates of all adjacent pairs become nearly equal, the
    coldest and hottest temperatures stay fixed and the ladder stays ordered; without
    adaptation the same ladder leaves the top pair almost never swapping."""
    lo, hi, mu, sig = _gauss_setup()
    T, W = 5, 32
    b0 = np.array([1.0, 0.9, 0.8, 0.7, 0.0])

    def rates(adapt):
        g = I.rng(61)
        x = lo[:, None] + (hi - lo)[:, None] * g.random((11, T * W))
        out = oracle.pt_gauss_loglike(x, mu, sig)
        x, out, _, _, bt = oracle.pt_run_gauss(x, out, T, W, b0, lo, hi, PROBS, 2.0, 11, 0, 3000, mu,
                                               sig, adapt=adapt, beta_trace=True)
        _, _, cnt, _, bt2 = oracle.pt_run_gauss(x, out, T, W, bt[-1], lo, hi, PROBS, 2.0, 11, 3000,
                                                1000, mu, sig, adapt=adapt, beta_trace=True)
        return cnt[8 * T + 1:9 * T] / cnt[9 * T + 1:10 * T], np.concatenate([bt, bt2])

    r0, _ = rates(None)
    assert r0[-1] < 0.05 and r0[:-1].min() > 0.8
    r, bt = rates((10.0, 200.0))
    assert r.min() > 0.1 and r.max() - r.min() < 0.06, r
    assert np.all(bt[:, 0] == 1.0) and np.all(bt[:, -1] == 0.0)
    assert np.all(np.diff(bt, axis=1) < 0)
