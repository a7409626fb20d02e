"""Pins of the oracle's wave frame against constructions that do not reuse its formulas
(R0 response, Sec. II A; the sky position and polarisation angle of Table I).

  * propagation direction: the template's group delay at the detector, minus the SSB time
    t(f), is the plane wave's arrival-time offset at the constellation's guiding centre,
    -n.c(t) for a source in direction n (a wavefront reaches the side facing the source
    first); n and c(t) are written here from spherical coordinates and the 1 AU orbit;
  * polarisation basis and angle: u, v built from the sky geometry (v along increasing
    latitude, u = n x v so that u x v = k), rotated right-handedly about k by psi with
    Rodrigues' formula, give P+ = u'u' - v'v' and Px = u'v' + v'u';
  * helicity: a face-on source (iota = 0) is circularly polarised, so rotating the
    polarisation frame (psi + a) is undone by advancing the orbital phase (phi + a), and
    for iota = pi by retarding it (phi - a): the sense of psi relative to phi.
A flipped propagation direction, a psi rotated the other way, or a mirrored basis fails them.
"""
import math

import numpy as np
import pytest

import mbh_inputs as I

AU_S = 1.495978707e11 / 299792458.0
YEAR = 31557600.0


def _source(lam, bet, tref, mt=1.0e6, psi=0.3, iota=0.7, phi=0.4):
    th = np.zeros(11)
    th[I.I_MT] = mt
    th[I.I_Q] = 0.5
    th[I.I_DL] = 10.0
    th[I.I_PHI] = phi
    th[I.I_IOTA] = iota
    th[I.I_LAM] = lam
    th[I.I_BETA] = bet
    th[I.I_PSI] = psi
    th[I.I_TREF] = tref
    return th


def _unit_to_source(lam, bet):
    return np.array([math.cos(bet) * math.cos(lam), math.cos(bet) * math.sin(lam), math.sin(bet)])


@pytest.mark.parametrize("dlam,bet", [(0.0, 0.0), (math.pi / 3, 0.4), (2.0, -0.7), (-2.5, 1.1)])
def test_arrival_time_at_the_detector(oracle, dlam, bet):
    """Group delay of the A and E templates minus the SSB time = -n.c(t) within the response's
    own delays (tens of seconds), against |n.c| of up to 499 s."""
    alpha = 1.0   # orbital angle at t_ref (not 0, so that a mirrored longitude shows)
    tref = alpha / (2 * math.pi) * YEAR
    th = _source(alpha + dlam, bet, tref)
    info = oracle.w0_info(th)
    t_obs = YEAR
    for frac in (0.5, 0.7, 0.9):
        f = frac * info["fmax"]
        h = 1e-9
        hp = oracle.template(th, np.array([f - h, f + h]), t_obs)
        _, _, t_ssb = oracle.w0(th, np.array([f]), t_obs)
        alpha_t = 2 * math.pi * t_ssb[0] / YEAR
        c = AU_S * np.array([math.cos(alpha_t), math.sin(alpha_t), 0.0])
        expect = -_unit_to_source(alpha + dlam, bet) @ c
        for ch in (0, 1):
            # h ~ e^{-i Phi}: group delay = d(-arg h)/df / 2 pi
            dphi = -np.angle(hp[ch, 1] * np.conj(hp[ch, 0]))
            tau = dphi / (2 * math.pi * 2 * h)
            assert abs((tau - t_ssb[0]) - expect) < 40.0, (frac, ch, tau - t_ssb[0], expect)


def _basis_from_geometry(lam, bet):
    """v: unit vector of increasing latitude; u = n x v, so that u x v = k = -n."""
    n = _unit_to_source(lam, bet)
    e = 1e-6
    dn = (_unit_to_source(lam, bet + e) - _unit_to_source(lam, bet - e)) / (2 * e)
    v = dn / np.linalg.norm(dn)
    u = np.cross(n, v)
    return u, v, -n


def _rotate(x, axis, ang):
    """Rodrigues: x rotated by ang right-handedly about the unit vector axis."""
    return (x * math.cos(ang) + np.cross(axis, x) * math.sin(ang)
            + axis * (axis @ x) * (1 - math.cos(ang)))


@pytest.mark.parametrize("lam,bet,psi", [(0.0, 0.0, math.pi / 8), (1.1, 0.5, 0.3), (4.0, -1.2, 2.9)])
def test_polarisation_tensors(oracle, lam, bet, psi):
    th = _source(lam, bet, 1e6, psi=psi)
    k, Pp, Pc, _, _ = oracle.wave_frame(th)
    u, v, kk = _basis_from_geometry(lam, bet)
    np.testing.assert_allclose(np.cross(u, v), kk, atol=1e-9)
    np.testing.assert_allclose(k, kk, atol=1e-9)
    up, vp = _rotate(u, kk, psi), _rotate(v, kk, psi)
    np.testing.assert_allclose(Pp, np.outer(up, up) - np.outer(vp, vp), atol=1e-9)
    np.testing.assert_allclose(Pc, np.outer(up, vp) + np.outer(vp, up), atol=1e-9)


def test_polarisation_closed_form_on_the_x_axis(oracle):
    """lambda = beta = 0, psi = pi/8: k = -x, u = -y, v = z; rotating by pi/8 about -x turns
    u toward v: u' = (0, -c, s), v' = (0, s, c) with c = cos(pi/8), s = sin(pi/8)."""
    th = _source(0.0, 0.0, 1e6, psi=math.pi / 8)
    k, Pp, Pc, _, _ = oracle.wave_frame(th)
    c, s = math.cos(math.pi / 8), math.sin(math.pi / 8)
    up, vp = np.array([0.0, -c, s]), np.array([0.0, s, c])
    np.testing.assert_allclose(k, [-1.0, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(Pp, np.outer(up, up) - np.outer(vp, vp), atol=1e-15)
    np.testing.assert_allclose(Pc, np.outer(up, vp) + np.outer(vp, up), atol=1e-15)
    # numerically: P+ = [[0,0,0],[0,1/sqrt2,-1/sqrt2],[0,-1/sqrt2,-1/sqrt2]]
    r = 1 / math.sqrt(2)
    np.testing.assert_allclose(Pp, [[0, 0, 0], [0, r, -r], [0, -r, -r]], atol=1e-15)
    np.testing.assert_allclose(Pc, [[0, 0, 0], [0, -r, -r], [0, -r, r]], atol=1e-15)


@pytest.mark.parametrize("iota,sense", [(0.0, 1.0), (math.pi, -1.0)])
def test_face_on_helicity(oracle, iota, sense):
    """Circular polarisation: the template at (psi + a, phi + sense a) equals the one at
    (psi, phi) to round-off for a face-on (sense +1) or face-off (sense -1) source."""
    g = I.grid_small(n=257, bin0=2000)
    f = oracle.freqs(g)
    th = _source(2.0, 0.3, 0.9 * g["t_obs"], mt=3e5, psi=0.4, iota=iota, phi=1.0)
    a = 0.37
    th2 = th.copy()
    th2[I.I_PSI] += a
    th2[I.I_PHI] += sense * a
    h1 = oracle.template(th, f, g["t_obs"])
    h2 = oracle.template(th2, f, g["t_obs"])
    assert np.abs(h1).max() > 0
    np.testing.assert_allclose(h2, h1, rtol=0, atol=1e-10 * np.abs(h1).max())
    # and the other pairing changes it (the test can see a wrong sense)
    th3 = th.copy()
    th3[I.I_PSI] += a
    th3[I.I_PHI] -= sense * a
    h3 = oracle.template(th3, f, g["t_obs"])
    assert np.abs(h3 - h1).max() > 0.1 * np.abs(h1).max()
