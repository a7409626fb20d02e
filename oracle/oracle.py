"""Python face of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
import this module.  It loads oracle/libmbh_oracle.so (plain C, see
mbh_oracle.c for what each part follows) through ctypes and adds the small
amount of numpy glue the tests need: the grid, the Gaussian noise scaling of
Sec. II (Re and Im of n~ each N(0, S/(4 df)), so E|n~|^2 = S/(2 df)), and the
distance rescaling that puts an injection at a target optimal SNR
sqrt(<h|h>) (Sec. II, remark under Eq. 3; h scales as 1/D_L, Sec. II A).
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        lp = C.POINTER(C.c_long)
        u32p = C.POINTER(C.c_uint32)
        sig = {
            "oracle_w0": (None, [dp, C.c_double, dp, C.c_long, dp, dp, dp]),
            "oracle_w0_info": (None, [dp, dp]),
            "oracle_orbit": (None, [C.c_double, dp]),
            "oracle_wave_frame": (None, [dp, dp, dp, dp, dp, dp]),
            "oracle_link": (None, [C.c_double, dp, dp, dp, dp]),
            "oracle_link_td": (None, [dp, dp, dp, dp, dp, C.c_double, dp, dp, dp, C.c_long, dp]),
            "oracle_tdi": (None, [C.c_double, dp, dp]),
            "oracle_template": (None, [dp, C.c_double, dp, C.c_long, dp]),
            "oracle_template_xyz": (None, [dp, C.c_double, dp, C.c_long, dp, dp]),
            "oracle_template_batch": (None, [dp, C.c_long, C.c_double, C.c_double, C.c_long,
                                             C.c_double, dp]),
            "oracle_psd": (None, [dp, C.c_long, dp]),
            "oracle_inner": (C.c_double, [dp, dp, dp, C.c_long, C.c_double, C.c_int]),
            "oracle_direct": (None, [dp, C.c_long, C.c_double, C.c_double, C.c_long, C.c_double,
                                     dp, dp, dp]),
            "oracle_het_edges": (C.c_long, [dp, C.c_double, C.c_double, C.c_long, C.c_double,
                                            C.c_int, lp, lp]),
            "oracle_het_prepare": (C.c_long, [dp, C.c_double, C.c_double, C.c_long, C.c_double,
                                              dp, dp, C.c_int, lp, dp, dp, dp]),
            "oracle_het_contract": (None, [C.c_long, lp, C.c_double, C.c_double, dp, dp,
                                           C.c_double, dp, C.c_long, dp]),
            "oracle_het_loglike": (None, [dp, C.c_long, C.c_long, lp, C.c_double, C.c_double,
                                          C.c_double, dp, dp, C.c_double, dp]),
            "oracle_philox4x32_10": (None, [u32p, u32p, u32p]),
            "oracle_sylm": (None, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, dp]),
            "oracle_hm_mode": (None, [dp, C.c_double, dp, C.c_long, C.c_int, dp, dp, dp, dp, dp]),
            "oracle_template_hm": (None, [dp, C.c_double, dp, C.c_long, C.c_uint, dp]),
            "oracle_template_batch_hm": (None, [dp, C.c_long, C.c_double, C.c_double, C.c_long,
                                                C.c_double, C.c_uint, dp]),
            "oracle_direct_hm": (None, [dp, C.c_long, C.c_double, C.c_double, C.c_long, C.c_double,
                                        C.c_uint, dp, dp, dp]),
            "oracle_het_edges_hm": (C.c_long, [dp, C.c_double, C.c_double, C.c_long, C.c_double,
                                               C.c_uint, C.c_int, lp, lp]),
            "oracle_het_prepare_hm": (C.c_long, [dp, C.c_double, C.c_double, C.c_long, C.c_double,
                                                 C.c_uint, dp, dp, C.c_int, lp, dp, dp, dp]),
            "oracle_het_loglike_hm": (None, [dp, C.c_long, C.c_long, lp, C.c_double, C.c_double,
                                             C.c_double, C.c_uint, dp, dp, C.c_double, dp]),
            "oracle_pt_theta": (None, [dp, C.c_long, dp]),
            "oracle_pt_choice": (None, [C.c_uint64, C.c_uint64, C.c_int, C.c_long, C.c_long, dp,
                                        C.c_double, dp]),
            "oracle_pt_sky": (None, [dp, C.c_int, C.c_int]),
            "oracle_pt_run_het": (None, [dp, dp, C.c_long, C.c_long, dp, dp, dp, dp, C.c_double,
                                         C.c_uint64, C.c_uint64, C.c_long, C.c_long, lp,
                                         C.c_double, C.c_double, C.c_double, dp, dp, C.c_double,
                                         lp, C.c_double, C.c_double]),
            "oracle_pt_run_gauss": (None, [dp, dp, C.c_long, C.c_long, dp, dp, dp, dp, C.c_double,
                                           C.c_uint64, C.c_uint64, C.c_long, dp, dp, lp, dp,
                                           C.c_double, C.c_double, dp]),
            "oracle_pt_gauss_loglike": (None, [dp, C.c_long, dp, dp, dp]),
            "oracle_pt_run_direct": (None, [dp, dp, C.c_long, C.c_long, dp, dp, dp, dp, C.c_double,
                                            C.c_uint64, C.c_uint64, C.c_long, C.c_double,
                                            C.c_double, C.c_long, C.c_double, C.c_uint, dp, dp,
                                            lp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _l(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_long))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def freqs(grid: dict) -> np.ndarray:
    return grid["f0"] + np.arange(grid["n"], dtype=np.float64) * grid["df"]


# ---- W0 -------------------------------------------------------------------
def w0(theta, f, t_obs):
    th, f = _f64(theta), _f64(f)
    n = f.size
    amp, psi, tf = np.empty(n), np.empty(n), np.empty(n)
    lib().oracle_w0(_d(th), t_obs, _d(f), n, _d(amp), _d(psi), _d(tf))
    return amp, psi, tf


W0_INFO_KEYS = ("M", "eta", "fc", "fcut", "fmax", "psi_max", "dpsi_max", "amp0", "dist")


def w0_info(theta) -> dict:
    out = np.empty(25)
    lib().oracle_w0_info(_d(_f64(theta)), _d(out))
    info = dict(zip(W0_INFO_KEYS, out[:9]))
    info["alpha"] = out[9:17].copy()
    info["alpha_log"] = out[17:25].copy()
    return info


# ---- R0 -------------------------------------------------------------------
def orbit(t: float) -> np.ndarray:
    p = np.empty(9)
    lib().oracle_orbit(float(t), _d(p))
    return p.reshape(3, 3)


def wave_frame(theta):
    k, Pp, Pc, Kp, Kc = np.empty(3), np.empty(9), np.empty(9), np.empty(2), np.empty(2)
    lib().oracle_wave_frame(_d(_f64(theta)), _d(k), _d(Pp), _d(Pc), _d(Kp), _d(Kc))
    return k, Pp.reshape(3, 3), Pc.reshape(3, 3), complex(*Kp), complex(*Kc)


def link(f, k, ps, pr) -> complex:
    G = np.empty(2)
    lib().oracle_link(float(f), _d(_f64(k)), _d(_f64(ps)), _d(_f64(pr)), _d(G))
    return complex(G[0], G[1])


def link_td(k, Pp, Pc, ps, pr, f0, ap: complex, ac: complex, t) -> np.ndarray:
    t = _f64(t)
    y = np.empty(t.size)
    lib().oracle_link_td(_d(_f64(k)), _d(_f64(Pp).ravel()), _d(_f64(Pc).ravel()), _d(_f64(ps)),
                         _d(_f64(pr)), float(f0), _d(_f64([ap.real, ap.imag])),
                         _d(_f64([ac.real, ac.imag])), _d(t), t.size, _d(y))
    return y


def tdi(f, y6) -> tuple[np.ndarray, np.ndarray]:
    y = _c128(y6).view(np.float64)
    out = np.empty(12)
    lib().oracle_tdi(float(f), _d(np.ascontiguousarray(y)), _d(out))
    z = out.view(np.complex128)
    return z[:3].copy(), z[3:].copy()


def template(theta, f, t_obs) -> np.ndarray:
    """A, E, T template, shape (3, n) complex128."""
    f = _f64(f)
    h = np.empty((3, f.size), dtype=np.complex128)
    lib().oracle_template(_d(_f64(theta)), t_obs, _d(f), f.size, _d(h.view(np.float64)))
    return h


def template_xyz(theta, f, t_obs):
    f = _f64(f)
    h = np.empty((3, f.size), dtype=np.complex128)
    x = np.empty((3, f.size), dtype=np.complex128)
    lib().oracle_template_xyz(_d(_f64(theta)), t_obs, _d(f), f.size, _d(h.view(np.float64)),
                              _d(x.view(np.float64)))
    return h, x


def template_batch(theta, grid, modes: int = 1) -> np.ndarray:
    """Templates on the grid for SoA theta (11, W): shape (W, 3, n) complex128."""
    th = np.ascontiguousarray(_f64(theta))
    W = th.shape[1]
    h = np.empty((W, 3, grid["n"]), dtype=np.complex128)
    lib().oracle_template_batch_hm(_d(th), W, grid["f0"], grid["df"], grid["n"], grid["t_obs"],
                                   int(modes), _d(h.view(np.float64)))
    return h


# ---- higher harmonics (W0-HM) ---------------------------------------------------
HM_MODES = ((2, 2), (3, 3), (4, 4), (2, 1), (3, 2), (4, 3))   # bit b of a mode mask
HM_ALL = 0x3F


def template_hm(theta, f, t_obs, modes: int) -> np.ndarray:
    f = _f64(f)
    h = np.empty((3, f.size), dtype=np.complex128)
    lib().oracle_template_hm(_d(_f64(theta)), t_obs, _d(f), f.size, int(modes),
                             _d(h.view(np.float64)))
    return h


def hm_mode(theta, f, t_obs, b: int):
    """Mode b alone: (|h_lm| without the mode factor, Psi_lm, t_lm, H_lm complex)."""
    f = _f64(f)
    n = f.size
    amp, psi, tf, hr, hi = (np.empty(n) for _ in range(5))
    lib().oracle_hm_mode(_d(_f64(theta)), t_obs, _d(f), n, int(b), _d(amp), _d(psi), _d(tf),
                         _d(hr), _d(hi))
    return amp, psi, tf, hr + 1j * hi


def sylm(s: int, l: int, m: int, theta: float, phi: float) -> complex:
    out = np.empty(2)
    lib().oracle_sylm(s, l, m, float(theta), float(phi), _d(out))
    return complex(out[0], out[1])


# ---- PSD, noise, inner products ---------------------------------------------
def psd(f) -> np.ndarray:
    f = _f64(f)
    S = np.empty((3, f.size))
    lib().oracle_psd(_d(f), f.size, _d(S))
    return S


def noise(S: np.ndarray, df: float, z: np.ndarray) -> np.ndarray:
    """Noise realisation from standard normals z (3, n, 2): Re, Im ~ N(0, S/(4 df))."""
    sig = np.sqrt(S / (4.0 * df))
    return sig * (z[..., 0] + 1j * z[..., 1])


def inner(a, b, S, df, compensated=False) -> float:
    a, b, S = _c128(a), _c128(b), _f64(S)
    n = a.shape[-1]
    return lib().oracle_inner(_d(a.view(np.float64)), _d(b.view(np.float64)), _d(S), n, df,
                              1 if compensated else 0)


def snr_distance(theta, grid, snr_target, S=None) -> float:
    """D_L (Gpc) that gives optimal SNR sqrt(<h|h>) = snr_target; h ~ 1/D_L."""
    f = freqs(grid)
    if S is None:
        S = psd(f)
    th = _f64(theta).copy()
    th[4] = 1.0
    h = template(th, f, grid["t_obs"])
    rho1 = math.sqrt(inner(h, h, S, grid["df"]))
    return rho1 / snr_target


def make_data(theta_inj, grid, z=None, S=None):
    """d = s + n on the grid (noise omitted when z is None); returns (d, S)."""
    f = freqs(grid)
    if S is None:
        S = psd(f)
    d = template(theta_inj, f, grid["t_obs"])
    if z is not None:
        d = d + noise(S, grid["df"], z)
    return np.ascontiguousarray(d), S


def direct(theta, grid, d, S, modes: int = 1) -> np.ndarray:
    """(3, W): lnL, <d|h>, <h|h> (Eqs. 2-3); templates of the modes of the mask."""
    th = _f64(theta)
    if th.ndim == 1:
        th = th[:, None]
    th = np.ascontiguousarray(th)
    W = th.shape[1]
    out = np.empty(3 * W)
    lib().oracle_direct_hm(_d(th), W, grid["f0"], grid["df"], grid["n"], grid["t_obs"],
                           int(modes), _d(_c128(d).view(np.float64)), _d(_f64(S)), _d(out))
    return out.reshape(3, W)


# ---- heterodyne ---------------------------------------------------------------
def het_edges(theta0, grid, nbins, modes: int = 1):
    edges = np.empty(nbins + 1, dtype=np.int64)
    band = np.empty(2, dtype=np.int64)
    E = lib().oracle_het_edges_hm(_d(_f64(theta0)), grid["f0"], grid["df"], grid["n"],
                                  grid["t_obs"], int(modes), nbins, _l(edges), _l(band))
    return (edges[:E + 1].copy() if E > 0 else edges[:0].copy()), band


def het_prepare(theta0, grid, d, S, nbins, modes: int = 1) -> dict:
    edges = np.empty(nbins + 1, dtype=np.int64)
    summ = np.empty(nbins * 3 * 6)
    h0e = np.empty((nbins + 1) * 3 * 2)
    dd = np.empty(1)
    E = lib().oracle_het_prepare_hm(_d(_f64(theta0)), grid["f0"], grid["df"], grid["n"],
                                    grid["t_obs"], int(modes), _d(_c128(d).view(np.float64)),
                                    _d(_f64(S)), nbins, _l(edges), _d(summ), _d(h0e), _d(dd))
    if E < 1:
        raise ValueError("empty heterodyne band")
    return dict(E=int(E), edges=edges[:E + 1].copy(),
                summary=summ[:E * 18].reshape(E, 3, 6).copy(),
                h0e=h0e[:(E + 1) * 6].view(np.complex128).reshape(E + 1, 3).copy(),
                dd=float(dd[0]), grid=dict(grid), modes=int(modes))


def het_contract(ref: dict, he: np.ndarray) -> np.ndarray:
    """he: (W, E+1, 3) template values at the edges."""
    he = _c128(he)
    W = he.shape[0]
    out = np.empty(3 * W)
    g = ref["grid"]
    lib().oracle_het_contract(ref["E"], _l(ref["edges"]), g["f0"], g["df"],
                              _d(_f64(ref["summary"]).ravel()), _d(_c128(ref["h0e"]).view(np.float64)),
                              ref["dd"], _d(he.view(np.float64)), W, _d(out))
    return out.reshape(3, W)


def het_loglike(theta, ref: dict) -> np.ndarray:
    th = _f64(theta)
    if th.ndim == 1:
        th = th[:, None]
    th = np.ascontiguousarray(th)
    W = th.shape[1]
    out = np.empty(3 * W)
    g = ref["grid"]
    lib().oracle_het_loglike_hm(_d(th), W, ref["E"], _l(ref["edges"]), g["f0"], g["df"],
                                g["t_obs"], int(ref.get("modes", 1)),
                                _d(_f64(ref["summary"]).ravel()),
                                _d(_c128(ref["h0e"]).view(np.float64)), ref["dd"], _d(out))
    return out.reshape(3, W)


def threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


# ---- parallel-tempered ensemble sampler (Sec. III) ------------------------------
PT_KINDS = ("stretch", "sky_all", "sky_lon", "sky_lat")


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr (n, 4) uint32 under key (2,) uint32: (n, 4) uint32."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    u32p = C.POINTER(C.c_uint32)
    for i in range(ctr.shape[0]):
        lib().oracle_philox4x32_10(ctr[i].ctypes.data_as(u32p), key.ctypes.data_as(u32p),
                                   out[i].ctypes.data_as(u32p))
    return out


def pt_theta(x) -> np.ndarray:
    """theta (11, n) of sampler coordinates x (11, n)."""
    x = np.ascontiguousarray(_f64(x))
    th = np.empty_like(x)
    lib().oracle_pt_theta(_d(x), x.shape[1], _d(th))
    return th


def pt_choice(seed, step, half, item, W, probs, a=2.0) -> dict:
    out = np.empty(5)
    lib().oracle_pt_choice(seed, step, half, item, W, _d(_f64(probs)), a, _d(out))
    return dict(kind=int(out[0]), j=int(out[1]), z=float(out[2]), n=int(out[3]), m=int(out[4]))


def pt_sky(x, n, m) -> np.ndarray:
    v = _f64(x).copy()
    lib().oracle_pt_sky(_d(v), int(n), int(m))
    return v


def _pt_common(x, out, betas, lo, hi, probs):
    x = np.ascontiguousarray(_f64(x)).copy()
    out = np.ascontiguousarray(_f64(out)).copy()
    return x, out, _f64(betas).copy(), _f64(lo), _f64(hi), _f64(probs)


def pt_run_het(x, out, T, W, betas, lo, hi, probs, a, seed, step0, n_iter, ref: dict,
               adapt=None, return_betas=False):
    """n_iter sampler iterations with the heterodyned likelihood; returns (x, out, counters)
    (and the final ladder with return_betas).  adapt = (nu, n0) adapts the ladder."""
    x, out, betas, lo, hi, probs = _pt_common(x, out, betas, lo, hi, probs)
    cnt = np.zeros(10 * T, dtype=np.int64)
    g = ref["grid"]
    nu, n0 = adapt if adapt else (0.0, 0.0)
    lib().oracle_pt_run_het(_d(x), _d(out), T, W, _d(betas), _d(lo), _d(hi), _d(probs), a,
                            seed, step0, n_iter, ref["E"], _l(ref["edges"]), g["f0"], g["df"],
                            g["t_obs"], _d(_f64(ref["summary"]).ravel()),
                            _d(_c128(ref["h0e"]).view(np.float64)), ref["dd"], _l(cnt),
                            float(nu), float(n0))
    return (x, out, cnt, betas) if return_betas else (x, out, cnt)


def pt_run_direct(x, out, T, W, betas, lo, hi, probs, a, seed, step0, n_iter, grid, d, S,
                  modes: int = 1):
    """n_iter sampler iterations with the direct likelihood; returns (x, out, counters)."""
    x, out, betas, lo, hi, probs = _pt_common(x, out, betas, lo, hi, probs)
    cnt = np.zeros(10 * T, dtype=np.int64)
    lib().oracle_pt_run_direct(_d(x), _d(out), T, W, _d(betas), _d(lo), _d(hi), _d(probs), a,
                               seed, step0, n_iter, grid["f0"], grid["df"], grid["n"],
                               grid["t_obs"], int(modes), _d(_c128(d).view(np.float64)),
                               _d(_f64(S)), _l(cnt))
    return x, out, cnt


def pt_run_gauss(x, out, T, W, betas, lo, hi, probs, a, seed, step0, n_iter, mu, sigma,
                 trace=False, adapt=None, beta_trace=False):
    """The sampler on a diagonal Gaussian target in x; returns (x, out, counters, trace),
    plus the ladder after every iteration with beta_trace.  adapt = (nu, n0)."""
    x, out, betas, lo, hi, probs = _pt_common(x, out, betas, lo, hi, probs)
    cnt = np.zeros(10 * T, dtype=np.int64)
    tr = np.empty((n_iter, 11, T * W)) if trace else None
    bt = np.empty((n_iter, T)) if beta_trace else None
    nu, n0 = adapt if adapt else (0.0, 0.0)
    lib().oracle_pt_run_gauss(_d(x), _d(out), T, W, _d(betas), _d(lo), _d(hi), _d(probs), a,
                              seed, step0, n_iter, _d(_f64(mu)), _d(_f64(sigma)), _l(cnt),
                              _d(tr) if trace else None, float(nu), float(n0),
                              _d(bt) if beta_trace else None)
    return (x, out, cnt, tr, bt) if beta_trace else (x, out, cnt, tr)


def pt_gauss_loglike(x, mu, sigma) -> np.ndarray:
    x = np.ascontiguousarray(_f64(x))
    out = np.empty(3 * x.shape[1])
    lib().oracle_pt_gauss_loglike(_d(x), x.shape[1], _d(_f64(mu)), _d(_f64(sigma)), _d(out))
    return out.reshape(3, -1)
