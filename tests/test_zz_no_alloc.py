"""direct_loglike_stored_noalloc: the stored-template direct likelihood for callers
that cannot allocate device memory (fixed budgets owned by another framework,
callbacks that must not enter the allocator).  Called through the C ABI and
compared with direct_loglike_stored, which takes its scratch from cudaMallocAsync,
on two calls in a row.  This file is collected last."""
import ctypes

import numpy as np
import pytest

import mbh_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01064_b300 import mbhlike as M
    from paper_2111_01064_b300 import workloads as WL
    g = I.grid_month()
    src = WL.source_for(0, g)
    th = WL.walkers(src.theta_inj, 13, 0, lo=1e-5, hi=1e-3)
    return M, WL, g, src, th


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_noalloc_matches_allocating_entry_point(case, prec):
    import torch
    M, WL, g, src, th = case
    h = M.template_batch(g, WL.to_dev(th), prec)
    ref = M.direct_loglike_stored(src.data, h, prec).cpu().numpy()
    for _ in range(2):
        out = torch.full((3, th.shape[1]), float("nan"), dtype=torch.float64, device="cuda")
        M.direct_loglike_stored_noalloc(src.data, h, prec, out=out)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-9)


def test_noalloc_rejects_batches_beyond_its_buffer(case):
    """Checked on the host before anything is queued (the pointers are never used)."""
    M, WL, g, src, th = case
    L = M.lib()
    st = L.direct_loglike_stored_noalloc(src.data.handle, None, 10_000_000, 0, None, None)
    assert st == 1
    msg = L.mbh_last_error().decode()
    assert "static buffer holds" in msg and str(8 << 20) in msg


def test_noalloc_limit_on_the_year_grid(case):
    """The documented limit on the 1-yr grid (1,051,920 points): large batches take
    ceil(n / 2^18) = 5 grid chunks of partial sums, 16 bytes per (template, chunk), so the
    8 MiB buffer holds W = 8 MiB / 80 B = 104857 templates.  Checked through the C ABI with
    NULL buffers: W = 104857 passes the size check and stops at the NULL-buffer check (nothing
    is queued), W = 104858 and 104861 are refused for their size."""
    import torch
    M, WL, g, src, th = case
    gy = I.grid_year()
    psd = M.mbh_psd_aet(gy)
    data = M.Data(gy, torch.zeros((3, gy["n"]), dtype=torch.complex128, device="cuda"), psd)
    L = M.lib()
    w_max = (8 << 20) // (16 * 5)
    assert w_max == 104857
    assert L.direct_loglike_stored_noalloc(data.handle, None, w_max, 0, None, None) == 1
    assert "NULL buffer" in L.mbh_last_error().decode()
    for w in (w_max + 1, w_max + 4):
        assert L.direct_loglike_stored_noalloc(data.handle, None, w, 0, None, None) == 1
        msg = L.mbh_last_error().decode()
        assert "static buffer holds" in msg and f"W={w}" in msg and "5 chunks" in msg, msg
