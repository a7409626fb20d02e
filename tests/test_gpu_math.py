"""The library's own float32 device math (used on the mixed-precision hot path) against
float64 references of the same float32 inputs and against CUDA's sin/cos."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01064_b300 import mbhlike
    mbhlike.lib()
    return mbhlike


def test_sincos_small(M):
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-8, 8, 1 << 20), rng.uniform(-1e-3, 1e-3, 1 << 16),
                        np.float32([0.0, np.pi / 4, -np.pi / 2, np.pi, 3 * np.pi / 2, 6.0])]).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    s, c = M.mbh_selftest_math(0, xt)
    s, c = s.cpu().numpy().astype(np.float64), c.cpu().numpy().astype(np.float64)
    xd = x.astype(np.float64)
    assert np.max(np.abs(s - np.sin(xd))) <= 3e-7
    assert np.max(np.abs(c - np.cos(xd))) <= 3e-7
    small = np.abs(xd) < 1e-3
    assert np.max(np.abs(s[small] - np.sin(xd[small])) / np.maximum(np.abs(xd[small]), 1e-30)) <= 2e-7
    # as close to the float64 values as CUDA's own sinf/cosf
    ts, tc = torch.sin(xt).double().cpu().numpy(), torch.cos(xt).double().cpu().numpy()
    assert np.max(np.abs(s - np.sin(xd))) <= 3.0 * np.max(np.abs(ts - np.sin(xd))) + 1e-8
    assert np.max(np.abs(c - np.cos(xd))) <= 3.0 * np.max(np.abs(tc - np.cos(xd))) + 1e-8


def test_sinc(M):
    import torch
    x = np.linspace(-3.0, 3.0, 600001).astype(np.float32)
    got = M.mbh_selftest_math(1, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    xd = x.astype(np.float64)
    ref = np.where(xd == 0, 1.0, np.sin(xd) / np.where(xd == 0, 1.0, xd))
    assert np.max(np.abs(got - ref)) <= 2e-7


def test_sinc_difference_relative(M):
    import mpmath as mp
    import torch
    rng = np.random.default_rng(2)
    x = rng.uniform(1e-5, 1.9, 2000).astype(np.float32)
    k = rng.uniform(-1, 1, 2000).astype(np.float32)
    got = M.mbh_selftest_math(2, torch.from_numpy(x).cuda(), torch.from_numpy(k).cuda()).cpu().numpy()
    mp.mp.dps = 40
    for i in range(0, 2000, 10):
        X, K = mp.mpf(float(x[i])), mp.mpf(float(k[i]))
        ref = float(mp.sinc(X * (1 + K)) - mp.sinc(X * (1 - K)))
        if max(abs(X * (1 + K)), abs(X * (1 - K))) < 2:     # series branch: relative accuracy
            assert abs(got[i] - ref) <= 1e-6 * abs(ref) + 1e-12, (x[i], k[i], got[i], ref)
        else:                                                  # plain difference of O(1) values
            assert abs(got[i] - ref) <= 3e-7, (x[i], k[i], got[i], ref)


def test_short_sinc_forms(M):
    """The four-term series used by the response below x = 0.1 agree with the float64
    values to float32 rounding over their whole range (|x| < 0.2; x < 0.1 with |k| <= 1)."""
    import mpmath as mp
    import torch
    x = np.linspace(-0.2, 0.2, 40001).astype(np.float32)
    got = M.mbh_selftest_math(3, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    xd = x.astype(np.float64)
    ref = np.where(xd == 0, 1.0, np.sin(xd) / np.where(xd == 0, 1.0, xd))
    assert np.max(np.abs(got - ref)) <= 1.2e-7
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.uniform(1e-5, 0.1, 1500), np.full(100, 0.0999999)]).astype(np.float32)
    ks = np.concatenate([rng.uniform(-1, 1, 1500), rng.choice([-1.0, 1.0], 100)]).astype(np.float32)
    got = M.mbh_selftest_math(4, torch.from_numpy(xs).cuda(), torch.from_numpy(ks).cuda()).cpu().numpy()
    full = M.mbh_selftest_math(2, torch.from_numpy(xs).cuda(), torch.from_numpy(ks).cuda()).cpu().numpy()
    mp.mp.dps = 40
    for i in range(0, 1600, 4):
        X, K = mp.mpf(float(xs[i])), mp.mpf(float(ks[i]))
        ref = float(mp.sinc(X * (1 + K)) - mp.sinc(X * (1 - K)))
        assert abs(got[i] - ref) <= 1e-6 * abs(ref) + 1e-14, (xs[i], ks[i], got[i], ref)
        assert abs(got[i] - full[i]) <= 1e-6 * abs(ref) + 1e-14
    with pytest.raises(M.MBHError):
        M.mbh_selftest_math(7, torch.from_numpy(xs).cuda())


def _split2(v):
    hi = v.astype(np.float32)
    return hi, (v - hi.astype(np.float64)).astype(np.float32)


def test_df_sincos_unnormalised(M):
    """The double-float sine and cosine - 1 of the extended kernels (kind 5) against 40-digit
    values of the same inputs: small angles, |x| <= pi and |x| ~ 1e6, with low words of up to 8
    ulps of the high word (lazy arithmetic after a cancellation leaves such pairs).  Bound: 5e-11
    (the series' float32 a^3 term at |a| <= 0.1, directly or after the reduction to within pi/32)
    plus |x| 2^-46 at large |x| (the reduction's rounding of the argument's low word)."""
    import mpmath as mp
    import torch
    rng = np.random.default_rng(7)
    hi = np.concatenate([rng.uniform(-0.19, 0.19, 400), rng.uniform(-3.2, 3.2, 400),
                         rng.uniform(-2e6, 2e6, 400)]).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (rng.integers(-16, 17, hi.size) * 0.5 * ulp).astype(np.float32)
    x = np.ascontiguousarray(np.stack([hi, lo], 1))
    s, c = M.mbh_selftest_math(5, torch.from_numpy(x).cuda())
    s, c = s.cpu().numpy(), c.cpu().numpy()
    mp.mp.dps = 40
    worst = 0.0
    for i in range(hi.size):
        xv = mp.mpf(float(hi[i])) + mp.mpf(float(lo[i]))
        es = abs(mp.mpf(float(s[i, 0])) + mp.mpf(float(s[i, 1])) - mp.sin(xv))
        ec = abs(mp.mpf(float(c[i, 0])) + mp.mpf(float(c[i, 1])) - (mp.cos(xv) - 1))
        bound = 5e-11 + abs(float(xv)) * 2.0 ** -46
        worst = max(worst, float(max(es, ec)) / bound)
        assert es <= bound and ec <= bound, (float(xv), float(es), float(ec))
    print("df sincos worst error / bound", worst)


def test_df_mul_mod2pi(M):
    """x y mod 2 pi (kind 6) for a double-float x (frequencies 1e-5..0.05 Hz) and a
    triple-float y (1e6..3e8: the time coefficient 2 pi t_ref of the absolute phase) against
    the exact product: within 1e-13 after the whole turns are removed, with no bias."""
    import mpmath as mp
    import torch
    rng = np.random.default_rng(8)
    n = 2000
    a = np.exp(rng.uniform(np.log(1e-5), np.log(0.05), n))
    b = np.exp(rng.uniform(np.log(1e6), np.log(3e8), n))
    ahi, alo = _split2(a)
    bhi, blo = _split2(b)
    bx = (b - bhi.astype(np.float64) - blo.astype(np.float64)).astype(np.float32)
    x = np.ascontiguousarray(np.stack([ahi, alo], 1))
    y = np.ascontiguousarray(np.stack([bhi, blo, bx], 1))
    r = M.mbh_selftest_math(6, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
    mp.mp.dps = 50
    two_pi = 2 * mp.pi
    errs = np.empty(n)
    for i in range(n):
        exact = (mp.mpf(float(ahi[i])) + mp.mpf(float(alo[i]))) * (mp.mpf(float(bhi[i])) + mp.mpf(float(blo[i]))
                                                                    + mp.mpf(float(bx[i])))
        got = mp.mpf(float(r[i, 0])) + mp.mpf(float(r[i, 1]))
        turns = mp.nint((exact - got) / two_pi)
        errs[i] = float(got - (exact - turns * two_pi))
        assert abs(got) < 8
    print("mod 2 pi product: max error", np.abs(errs).max(), "mean", errs.mean())
    assert np.abs(errs).max() <= 1e-13
    assert abs(errs.mean()) <= 1e-14
