"""Pins of the oracle's higher-harmonic stand-in "W0-HM" (Sec. II A, Eqs. 7-9: the template is
the sum over modes (l,m) of the transfer at t_lm(f) times h_lm; t_lm from the SPA, Eq. 8).

What fixes it independently of its own code: the spin-weighted harmonics against their
orthonormality, pole values, conjugation symmetry and textbook closed forms; each mode's
phase, time and amplitude against the stationary-phase relations t = Psi'/(2 pi) and
|h~| ~ a(t) sqrt(Psi''); the (2,2) limit against W0; linearity in the modes; the heterodyne
identity at the reference.  The leading post-Newtonian mode factors H_lm (literature values)
and parity with PhenomHM itself are unpinned."""
import math

import numpy as np
import pytest

import mbh_inputs as I


def test_sylm_orthonormal(oracle):
    x, wx = np.polynomial.legendre.leggauss(48)
    nphi = 24
    phis = 2 * math.pi * np.arange(nphi) / nphi
    lm = [(l, m) for l in (2, 3, 4) for m in range(-l, l + 1)]
    Y = np.array([[[oracle.sylm(-2, l, m, math.acos(c), p) for p in phis] for c in x] for l, m in lm])
    G = np.einsum("atp,btp,t->ab", Y, Y.conj(), wx) * (2 * math.pi / nphi)
    assert np.abs(G - np.eye(len(lm))).max() < 1e-12


def test_sylm_poles_symmetry_closed_forms(oracle):
    for l in (2, 3, 4):
        for m in range(-l, l + 1):
            y0 = oracle.sylm(-2, l, m, 0.0, 0.4)
            if m == 2:   # only m = -s survives at theta = 0
                assert abs(y0) == pytest.approx(math.sqrt((2 * l + 1) / (4 * math.pi)), rel=1e-14)
            else:
                assert abs(y0) < 1e-15
            th, ph = 1.1, 0.7
            # conj(sY_lm) = (-1)^(s+m) (-s)Y_{l,-m}
            assert np.conj(oracle.sylm(-2, l, m, th, ph)) == pytest.approx(
                (-1) ** m * oracle.sylm(2, l, -m, th, ph), abs=1e-14)
    th, ph = 0.83, -0.4
    c = math.cos(th)
    assert oracle.sylm(-2, 2, 2, th, ph) == pytest.approx(
        math.sqrt(5 / (64 * math.pi)) * (1 + c) ** 2 * np.exp(2j * ph), rel=1e-14)
    assert oracle.sylm(-2, 2, -2, th, ph) == pytest.approx(
        math.sqrt(5 / (64 * math.pi)) * (1 - c) ** 2 * np.exp(-2j * ph), rel=1e-14)
    assert oracle.sylm(-2, 2, 1, th, ph) == pytest.approx(
        math.sqrt(5 / (16 * math.pi)) * math.sin(th) * (1 + c) * np.exp(1j * ph), rel=1e-14)


@pytest.fixture(scope="module")
def src():
    g = I.grid_month()
    th, _ = I.draw_source(I.rng(0), g["t_obs"], mt_range=(3e5, 3e5))
    th[I.I_Q] = 0.4
    return g, th


@pytest.mark.parametrize("b", range(6))
def test_mode_spa_relations(oracle, src, b):
    """t_lm = Psi_lm'/(2 pi) and |h_lm| / |h_22(2f/m)| = |H_lm| sqrt(Psi_lm''(f) / Psi_22''(2f/m))."""
    g, th = src
    m = oracle.HM_MODES[b][1]
    info = oracle.w0_info(th)
    f = np.geomspace(info["fmax"] * 0.05, info["fmax"] * 0.5, 7) * m / 2
    h = f * 1e-4
    fs = np.concatenate([f + k * h for k in (-2, -1, 0, 1, 2)])
    amp, psi, tf, H = oracle.hm_mode(th, fs, 1e12, b)
    P = psi.reshape(5, -1)
    d1 = (P[0] - 8 * P[1] + 8 * P[3] - P[4]) / (12 * h)
    d2 = (-P[0] + 16 * P[1] - 30 * P[2] + 16 * P[3] - P[4]) / (12 * h * h)
    t0 = tf.reshape(5, -1)[2]
    np.testing.assert_allclose(d1 / (2 * math.pi), t0, rtol=1e-7, atol=1e-3)
    f2 = 2 * f / m
    f2s = np.concatenate([f2 + k * (2 * h / m) for k in (-2, -1, 0, 1, 2)])
    a22, p22, t22, _ = oracle.hm_mode(th, f2s, 1e12, 0)
    Q = p22.reshape(5, -1)
    d2_22 = (-Q[0] + 16 * Q[1] - 30 * Q[2] + 16 * Q[3] - Q[4]) / (12 * (2 * h / m) ** 2)
    np.testing.assert_allclose(t22.reshape(5, -1)[2], t0, rtol=1e-12)   # same instant
    ratio = amp.reshape(5, -1)[2] / a22.reshape(5, -1)[2]
    np.testing.assert_allclose(ratio, np.sqrt(d2 / d2_22), rtol=1e-5)
    x = (math.pi * info["M"] * f2) ** (2 / 3)
    # mode factors vanish where they must: odd m at equal masses
    if m % 2 == 1:
        th1 = th.copy()
        th1[I.I_Q] = 1.0
        assert np.all(oracle.hm_mode(th1, f, 1e12, b)[3] == 0)
    Hc = H.reshape(5, -1)[2]
    assert x.max() < 1 and (np.all(Hc == 1) if b == 0 else np.all(np.abs(Hc) < 1))


def test_hm_22_limit_and_linearity(oracle, src):
    g, th = src
    f = oracle.freqs(g)
    th1 = th.copy()
    th1[I.I_Q] = 1.0    # (2,1) vanishes: the HM path with (2,2)+(2,1) must equal W0
    w0 = oracle.template(th1, f, g["t_obs"])
    hm = oracle.template_hm(th1, f, g["t_obs"], 0x1 | 0x8)
    assert np.abs(hm - w0).max() <= 1e-12 * np.abs(w0).max()
    assert np.abs(w0).max() > 0
    allm = oracle.template_hm(th, f, g["t_obs"], oracle.HM_ALL)
    parts = sum(oracle.template_hm(th, f, g["t_obs"], 1 << b) for b in range(6))
    assert np.abs(allm - parts).max() <= 1e-13 * np.abs(allm).max()
    for b in range(1, 6):   # every higher mode contributes ((4,3) is ~x^{3/2} smaller)
        assert np.abs(oracle.template_hm(th, f, g["t_obs"], 1 << b)).max() > 1e-5 * np.abs(w0).max()


def test_hm_band_and_het_identity(oracle):
    g = I.grid_month()
    th, snr = I.draw_source(I.rng(0), g["t_obs"])
    th[I.I_Q] = 0.3
    f = oracle.freqs(g)
    S = oracle.psd(f)
    th[I.I_DL] = oracle.snr_distance(th, g, snr, S)
    d = oracle.template_hm(th, f, g["t_obs"], oracle.HM_ALL)
    _, band22 = oracle.het_edges(th, g, 64)
    _, band = oracle.het_edges(th, g, 64, oracle.HM_ALL)
    assert band[0] <= band22[0] and band[1] >= band22[1]
    # noiseless data: direct lnL vanishes at the injection; heterodyne equals direct there
    out_d = oracle.direct(th[:, None], g, d, S, oracle.HM_ALL)
    assert abs(out_d[0, 0]) <= 1e-9 * out_d[2, 0]
    ref = oracle.het_prepare(th, g, d, S, 64, oracle.HM_ALL)
    out_h = oracle.het_loglike(th[:, None], ref)
    assert out_h[1, 0] == pytest.approx(out_d[1, 0], rel=1e-12)
    assert out_h[2, 0] == pytest.approx(out_d[2, 0], rel=1e-12)
    # a (2,2)-only template against higher-mode data fits worse than the full model
    out22 = oracle.direct(th[:, None], g, d, S, 1)
    assert out22[0, 0] < out_d[0, 0] - 1.0
