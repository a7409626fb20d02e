"""Pins of the oracle's W0 waveform (Sec. II A, Eq. 7 and the f_ref = f_max
convention) against results that do not come from the oracle's own formulas."""
import math

import numpy as np
import pytest
import sympy as sp

import mbh_inputs as I


def _theta(mt=1e6, q=0.5, a1=0.3, a2=-0.2, tref=2e6):
    th = np.array([mt, q, a1, a2, 1.0, 0.3, 0.8, 1.1, 0.2, 0.4, tref])
    return th


def test_fmax_is_argmax_f2A(oracle):
    """f_max = f_c sqrt(5/12) is where f^2 A(f) peaks (the f_ref convention)."""
    th = _theta()
    info = oracle.w0_info(th)
    f = np.geomspace(info["fmax"] / 3, info["fmax"] * 3, 200001)
    amp, _, _ = oracle.w0(th, f, 1e12)   # window wide enough to keep the support
    i = np.argmax(f * f * amp)
    assert abs(f[i] / info["fmax"] - 1) < 1e-4


def test_t_of_fmax_is_tref(oracle):
    th = _theta(tref=1.234567e6)
    info = oracle.w0_info(th)
    _, _, tf = oracle.w0(th, np.array([info["fmax"]]), 1e12)
    assert abs(tf[0] - th[10]) < 1e-9


def test_phase_derivative_is_2pi_t(oracle):
    """SPA (Eq. 8): dPsi/df = 2 pi t(f).  Five-point finite difference of the
    oracle's phase against its t(f)."""
    for mt in (1e5, 1e6, 1e7):
        th = _theta(mt=mt, tref=0.0)    # tref = 0 keeps Psi small for the difference
        info = oracle.w0_info(th)
        for x in (0.05, 0.2, 0.6, 1.0, 2.0):
            f0 = x * info["fmax"]
            h = f0 * 1e-4
            f = f0 + h * np.array([-2, -1, 0, 1, 2], dtype=float)
            _, psi, tf = oracle.w0(th, f, 1e12)
            fd = (psi[0] - 8 * psi[1] + 8 * psi[3] - psi[4]) / (12 * h)
            scale = max(abs(2 * math.pi * tf[2]), 1e-3 / f0)
            assert abs(fd - 2 * math.pi * tf[2]) / scale < 1e-7, (mt, x, fd, 2 * math.pi * tf[2])


def _taylorf2_from_energy_flux(eta_val):
    """TaylorF2 coefficients re-derived from the post-Newtonian binding energy
    E(v) and flux F(v) of a non-spinning binary (energy balance dE/dt = -F, SPA
    phase Psi = 2 pi f t - 2 phi), re-expanded to relative v^7.  Returns
    alpha_k (k = 0..7, constants of the v^5 and ln terms aside), alpha5_log,
    alpha6_log; the v^6 constant includes ln 4 and gamma_E from ln(16 v^2)."""
    v, L, eta = sp.symbols("v L eta", positive=True)
    pi, gE = sp.pi, sp.EulerGamma
    e2 = -sp.Rational(3, 4) - eta / 12
    e4 = -sp.Rational(27, 8) + sp.Rational(19, 8) * eta - eta**2 / 24
    e6 = (-sp.Rational(675, 64) + (sp.Rational(34445, 576) - sp.Rational(205, 96) * pi**2) * eta
          - sp.Rational(155, 96) * eta**2 - sp.Rational(35, 5184) * eta**3)
    f2 = -sp.Rational(1247, 336) - sp.Rational(35, 12) * eta
    f3 = 4 * pi
    f4 = -sp.Rational(44711, 9072) + sp.Rational(9271, 504) * eta + sp.Rational(65, 18) * eta**2
    f5 = (-sp.Rational(8191, 672) - sp.Rational(583, 24) * eta) * pi
    # ln(16 x) with x = v^2 -> ln 16 + 2 L, L = ln v
    f6 = (sp.Rational(6643739519, 69854400) + sp.Rational(16, 3) * pi**2
          - sp.Rational(1712, 105) * gE - sp.Rational(856, 105) * (sp.log(16) + 2 * L)
          + (-sp.Rational(134543, 7776) + sp.Rational(41, 48) * pi**2) * eta
          - sp.Rational(94403, 3024) * eta**2 - sp.Rational(775, 324) * eta**3)
    f7 = (-sp.Rational(16285, 504) + sp.Rational(214745, 1728) * eta
          + sp.Rational(193385, 3024) * eta**2) * pi
    # E = -eta M v^2/2 (1 + e2 v^2 + e4 v^4 + e6 v^6); dE/dv normalised by -eta M v
    num = 1 + 2 * e2 * v**2 + 3 * e4 * v**4 + 4 * e6 * v**6
    den = 1 + f2 * v**2 + f3 * v**3 + f4 * v**4 + f5 * v**5 + f6 * v**6 + f7 * v**7
    S = sp.series(num / den, v, 0, 8).removeO()
    S = sp.expand(S.subs(eta, eta_val))
    s = [S.coeff(v, k) for k in range(8)]
    alpha = {}
    for k in (0, 1, 2, 3, 4, 6, 7):
        sk = s[k]
        if k == 6:
            # s6 = c + cl L: integrate u^{-3}(c + cl ln u) and (c + cl ln u)
            c, cl = sk.coeff(L, 0), sk.coeff(L, 1)
            alpha[6] = -20 * c + 10 * cl
            alpha["6log"] = -20 * cl
        else:
            alpha[k] = 40 * sk / ((k - 8) * (k - 5))
    alpha["5log"] = -sp.Rational(40, 3) * s[5]
    return {key: float(sp.N(val, 30)) for key, val in alpha.items()}


@pytest.mark.parametrize("q", [1.0, 0.5, 0.1])
def test_pn_phase_coefficients_from_energy_balance(oracle, q):
    """Non-spinning TaylorF2 coefficients of W0 equal those re-derived from the
    binding energy and the flux (a different published set of numbers)."""
    th = _theta(q=q, a1=0.0, a2=0.0)
    info = oracle.w0_info(th)
    ref = _taylorf2_from_energy_flux(info["eta"])
    a, al = info["alpha"], info["alpha_log"]
    for k in (0, 1, 2, 3, 4, 6, 7):
        assert a[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-9), k
    assert al[5] == pytest.approx(ref["5log"], rel=1e-12)
    assert al[6] == pytest.approx(ref["6log"], rel=1e-12)
    for k in (0, 1, 2, 3, 4, 7):
        assert al[k] == 0.0


def test_spin_terms_against_symmetric_antisymmetric_form(oracle):
    """1.5PN spin-orbit and 2PN spin-spin terms against the chi_s/chi_a form:
    beta = 113/12 (chi_s + delta chi_a - 76 eta chi_s / 113), alpha_3 = -16 pi + 4 beta,
    sigma = 79/8 eta chi1 chi2, alpha_4 gets -10 sigma."""
    for q, a1, a2 in ((1.0, 0.5, 0.5), (0.3, 0.9, -0.4), (0.7, -0.8, 0.6)):
        th0 = _theta(q=q, a1=0.0, a2=0.0)
        th = _theta(q=q, a1=a1, a2=a2)
        i0, i1 = oracle.w0_info(th0), oracle.w0_info(th)
        eta = i1["eta"]
        delta = (1 - q) / (1 + q)      # (m1 - m2)/M
        cs, ca = 0.5 * (a1 + a2), 0.5 * (a1 - a2)
        beta = 113.0 / 12.0 * (cs + delta * ca - 76.0 * eta * cs / 113.0)
        sigma = 79.0 / 8.0 * eta * a1 * a2
        assert i1["alpha"][3] - i0["alpha"][3] == pytest.approx(4 * beta, rel=1e-12, abs=1e-13)
        assert i1["alpha"][4] - i0["alpha"][4] == pytest.approx(-10 * sigma, rel=1e-12, abs=1e-13)


def test_newtonian_amplitude(oracle):
    """|K+ A| at face-on inclination equals the Newtonian SPA amplitude
    sqrt(5/24) pi^{-2/3} Mc^{5/6} f^{-7/6} / D (G = c = 1, seconds) well below f_c."""
    th = _theta(mt=2e6, q=0.4, tref=1e11)   # keep t(f) inside the window
    th[6] = 0.0        # iota = 0
    info = oracle.w0_info(th)
    f = np.array([info["fc"] * 1e-3])
    amp, _, _ = oracle.w0(th, f, 1e12)
    assert amp[0] > 0
    _, _, _, Kp, _ = oracle.wave_frame(th)
    M, eta = info["M"], info["eta"]
    mc = eta ** 0.6 * M
    D = th[4] * 1e9 * 3.085677581491367e16 / 299792458.0
    newt = math.sqrt(5 / 24) * math.pi ** (-2 / 3) * mc ** (5 / 6) * f[0] ** (-7 / 6) / D
    assert abs(Kp) * amp[0] == pytest.approx(newt * math.exp(-(f[0] / info["fc"]) ** 2), rel=1e-12)


def test_amplitude_scales_as_inverse_distance(oracle):
    th = _theta()
    f = np.geomspace(1e-4, 1e-2, 7)
    a1, p1, t1 = oracle.w0(th, f, 1e12)
    th2 = th.copy(); th2[4] = 3.7
    a2, p2, t2 = oracle.w0(th2, f, 1e12)
    np.testing.assert_allclose(a2 * 3.7, a1, rtol=1e-14)
    np.testing.assert_array_equal(p1, p2)


def test_support_window(oracle):
    """A = 0 above f_cut = 0.2/M and where t(f) is outside [0, t_obs]."""
    th = _theta(mt=1e6, tref=3e5)
    info = oracle.w0_info(th)
    f = np.geomspace(1e-6, 2 * info["fcut"], 4001)
    amp, _, tf = oracle.w0(th, f, 1e6)
    inside = (f <= info["fcut"]) & (tf >= 0) & (tf <= 1e6)
    assert np.all(amp[~inside] == 0)
    assert np.all(amp[inside] > 0)
    assert inside.any() and (~inside).any()
