"""Pins of the oracle's R0 response (Sec. II A, Eqs. 4-6 and 9) and PSD
(remark under Eq. 3) against independent constructions."""
import math

import numpy as np
import pytest

C = 299792458.0
LS = 2.5e9 / C           # arm length in seconds
AU_S = 1.495978707e11 / C
YEAR = 31557600.0


def _theta(**kw):
    th = np.array([1e6, 0.5, 0.3, -0.2, 1.0, 0.3, 0.8, 1.1, 0.2, 0.4, 2e6])
    for i, v in kw.items():
        th[int(i)] = v
    return th


@pytest.mark.parametrize("t", [0.0, 1.3e6, 7.77e6, 2.5e7])
def test_orbit_rigid_equilateral(oracle, t):
    p = oracle.orbit(t)
    for i in range(3):
        for j in range(i + 1, 3):
            assert np.linalg.norm(p[i] - p[j]) == pytest.approx(LS, rel=1e-13)
    a = 2 * math.pi * t / YEAR
    np.testing.assert_allclose(p.mean(axis=0), AU_S * np.array([math.cos(a), math.sin(a), 0.0]),
                               rtol=0, atol=1e-9)
    nrm = np.cross(p[1] - p[0], p[2] - p[0])
    nrm /= np.linalg.norm(nrm)
    assert abs(abs(nrm[2]) - 0.5) < 1e-12      # plane at 60 degrees to the ecliptic
    np.testing.assert_allclose(oracle.orbit(t + YEAR), p, rtol=0, atol=1e-7)


def test_one_link_kernel_against_time_domain(oracle):
    """G(f) of the one-link kernel against a DFT of the time-domain Doppler
    response y(t) of a monochromatic wave with a frozen constellation."""
    th = _theta()
    k, Pp, Pc, _, _ = oracle.wave_frame(th)
    p = oracle.orbit(3.3e6)
    N, dt = 1 << 16, 1.0
    T = N * dt
    t = np.arange(N) * dt
    for m in (7, 655, 3001, 20011):
        f0 = m / T
        ap, ac = 0.7 - 0.2j, -0.3 + 0.9j
        for s, r in ((0, 1), (1, 0), (2, 0), (1, 2)):
            y = oracle.link_td(k, Pp, Pc, p[s], p[r], f0, ap, ac, t)
            Y = np.sum(y * np.exp(-2j * math.pi * m * np.arange(N) / N)) * dt
            n = (p[r] - p[s]) / LS
            nHn = n @ (0.5 * T * (ap * Pp + ac * Pc)) @ n
            G = oracle.link(f0, k, p[s], p[r])
            assert abs(Y - G * nHn) <= 1e-9 * abs(G * nHn), (m, s, r, Y, G * nHn)


def test_aet_orthonormal(oracle):
    f = np.geomspace(1e-4, 3e-2, 11)
    th = _theta(**{"10": 5e6})
    h, x = oracle.template_xyz(th, f, 1e8)
    np.testing.assert_allclose(np.sum(np.abs(h) ** 2, axis=0), np.sum(np.abs(x) ** 2, axis=0),
                               rtol=1e-13)


def test_long_wavelength_michelson_limit(oracle):
    """fL -> 0: X -> 8 pi^2 f^2 L^2 e^{-2 pi i f k.c} (F12 - F13) h22 with
    F_ij = n_ij.(P+ K+ + Px Kx).n_ij, and the error shrinks linearly with f."""
    th = _theta(**{"0": 1e7, "10": 1e12})
    k, Pp, Pc, Kp, Kc = oracle.wave_frame(th)
    errs = []
    for f in (1e-5, 1e-6):
        amp, psi, tf = oracle.w0(th, np.array([f]), 1e13)
        assert amp[0] > 0
        h22 = amp[0] * np.exp(-1j * psi[0])
        p = oracle.orbit(tf[0])
        c = p.mean(axis=0)
        Fm = Pp * Kp + Pc * Kc

        def F(i, j):
            n = (p[j] - p[i]) / LS
            return n @ Fm @ n
        pred = 8 * math.pi ** 2 * f ** 2 * LS ** 2 * np.exp(-2j * math.pi * f * (k @ c)) \
            * (F(0, 1) - F(0, 2)) * h22
        _, x = oracle.template_xyz(th, np.array([f]), 1e13)
        errs.append(abs(x[0, 0] / pred - 1))
    assert errs[0] < 3e-3
    assert errs[1] < 0.15 * errs[0]


def test_T_channel_suppressed_at_low_frequency(oracle):
    th = _theta(**{"10": 1e12})
    r = []
    for f in (1e-3, 1e-4, 1e-5):
        h = oracle.template(th, np.array([f]), 1e13)
        r.append(abs(h[2, 0]) / abs(h[0, 0]))
    assert r[1] < 0.2 * r[0] and r[2] < 0.2 * r[1]


def _tdi_matrix(oracle, f):
    """Coefficients of X, Y, Z, A, E, T in the six link responses."""
    M = np.zeros((6, 6), dtype=complex)
    for l in range(6):
        e = np.zeros(6, dtype=complex)
        e[l] = 1.0
        xyz, aet = oracle.tdi(f, e)
        M[:3, l] = xyz
        M[3:, l] = aet
    return M


# link order of y[6]: 1->2, 2->1, 2->3, 3->2, 3->1, 1->3 (0-based spacecraft)
_LINKS = [(0, 1), (1, 0), (1, 2), (2, 1), (2, 0), (0, 2)]


def test_psd_from_link_noise_through_tdi(oracle):
    """The analytic A, E, T PSD equals link-level noise pushed through the
    oracle's own TDI coefficients: independent OMS noise on each of the six
    links, and six test masses (i facing j) each entering y_{i->j} delayed by L
    and y_{j->i} undelayed with the same sign.  Cross-spectra vanish (A, E, T
    uncorrelated, Sec. II A)."""
    f = np.geomspace(2e-5, 5e-2, 23)
    S = oracle.psd(f)
    for i, fi in enumerate(f):
        M = _tdi_matrix(oracle, fi)[3:]           # A, E, T rows
        D = np.exp(-2j * math.pi * fi * LS)
        sacc = (3e-15) ** 2 * (1 + (4e-4 / fi) ** 2) * (1 + (fi / 8e-3) ** 4) / (2 * math.pi * fi * C) ** 2
        soms = (15e-12) ** 2 * (1 + (2e-3 / fi) ** 4) * (2 * math.pi * fi / C) ** 2
        cov = soms * (M @ M.conj().T)
        for (a, b) in ((0, 1), (1, 2), (2, 0)):
            la, lb = _LINKS.index((a, b)), _LINKS.index((b, a))
            for (s, r) in ((a, b), (b, a)):
                # test mass in s facing r
                v = np.zeros(6, dtype=complex)
                v[_LINKS.index((s, r))] += D
                v[_LINKS.index((r, s))] += 1.0
                col = M @ v
                cov = cov + sacc * np.outer(col, col.conj())
        np.testing.assert_allclose(np.diag(cov).real, S[:, i], rtol=1e-10)
        off = np.abs(cov - np.diag(np.diag(cov)))
        assert off.max() <= 1e-10 * np.abs(np.diag(cov)).max()


def test_psd_A_equals_E_and_T_small(oracle):
    f = np.geomspace(1e-5, 1e-1, 101)
    S = oracle.psd(f)
    np.testing.assert_array_equal(S[0], S[1])
    low = f < 1e-3
    assert np.all(S[2][low] < 1e-2 * S[0][low])
