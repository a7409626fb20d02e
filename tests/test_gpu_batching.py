"""Uneven multi-source batching (many sources with their own bin counts in one
launch), launch configurations, the autotuner and CUDA-graph replay.  A walker's
heterodyned lnL is a fixed-order computation of its own, so every launch shape must
give bit-identical results; a sample is also checked against the oracle."""
import numpy as np
import pytest

import mbh_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01064_b300 import mbhlike
    mbhlike.lib()
    return mbhlike


@pytest.fixture(scope="module")
def batch(M):
    from paper_2111_01064_b300 import workloads as WL
    return WL.uneven_batch(n_sources=12, walkers=(8, 256))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_f32"])
def test_launch_configurations(M, batch, prec):
    """For a given number of threads per walker G (which fixes the order in which a
    walker's bins are summed) every block size and persistent mode gives bit-identical
    results; different G agree to the last bits."""
    import torch
    th = torch.from_numpy(batch.theta).cuda()
    ref = M.het_loglike_batch(batch.refs, batch.offsets, th, prec).cpu().numpy()
    scale = np.abs(ref).max(axis=1, keepdims=True)
    extra = {2: (32,), 4: (32, 96, 160, 224), 8: (96, 160, 224), 16: (224,)} if prec == "mixed_f32" else {}
    for g in (1, 2, 4, 8, 16, 32):
        first = None
        for b in (0, 64, 128, 256) + extra.get(g, ()):
            if 0 < b < g:
                continue
            for pers in (0, 1):
                out = M.het_loglike_batch_cfg(batch.refs, batch.offsets, th, prec,
                                              M.het_config(g, b, pers)).cpu().numpy()
                if first is None:
                    first = out
                np.testing.assert_array_equal(out, first, err_msg=f"G={g} block={b} persistent={pers}")
        assert np.all(np.abs(first - ref) <= 1e-12 * scale), g


def test_uneven_batch_equals_per_source(M, batch):
    import torch
    th = torch.from_numpy(batch.theta).cuda()
    allg = M.het_loglike_batch(batch.refs, batch.offsets, th, "mixed").cpu().numpy()
    for s in range(len(batch.refs)):
        a, b = batch.offsets[s], batch.offsets[s + 1]
        one = M.het_loglike_batch([batch.refs[s]], [0, b - a],
                                  torch.from_numpy(np.ascontiguousarray(batch.theta[:, a:b])).cuda(),
                                  "mixed").cpu().numpy()
        np.testing.assert_array_equal(allg[:, a:b], one)


def test_uneven_batch_against_oracle(M, batch, oracle):
    """Two sources of the batch rebuilt on the oracle side from the same draws; their
    walkers' heterodyned lnL within the parity tolerances."""
    import torch
    th = torch.from_numpy(batch.theta).cuda()
    o64 = M.het_loglike_batch(batch.refs, batch.offsets, th, "fp64").cpu().numpy()
    omx = M.het_loglike_batch(batch.refs, batch.offsets, th, "mixed").cpu().numpy()
    g = I.grid_month()
    f = oracle.freqs(g)
    S = oracle.psd(f)
    for s in (0, 5):
        th_raw, snr = I.draw_source(I.rng(3, s), g["t_obs"])
        th0 = I.with_distance(th_raw, oracle.snr_distance(th_raw, g, snr, S))
        z = I.noise_normals(I.rng(3, 100 + s), g["n"])
        d, _ = oracle.make_data(th0, g, z, S)
        ref = oracle.het_prepare(th0, g, d, S, int(batch.bins[s]))
        assert ref["E"] == batch.refs[s].bins
        a, b = batch.offsets[s], batch.offsets[s + 1]
        wo = I.perturb(th0, I.perturbation(I.rng(3, 200 + s), b - a, 1e-5, 1e-3))
        out = oracle.het_loglike(wo, ref)
        scale = 0.5 * (ref["dd"] + np.abs(out[2]) + 2 * np.abs(out[1]))
        assert np.all(np.abs(o64[0, a:b] - out[0]) <= 1e-6 * scale)
        d = np.abs(omx[0, a:b] - out[0])
        print(f"uneven batch source {s}: mixed vs oracle p50/max", np.median(d), d.max())
        assert d.max() <= 1e-3


def test_autotune_returns_a_valid_configuration(M, batch):
    import torch
    th = torch.from_numpy(batch.theta).cuda()
    cfg, ms = M.mbh_het_autotune(batch.refs, batch.offsets, th, "mixed", reps=1)
    assert cfg.threads_per_walker in (1, 2, 4, 8, 16, 32) and cfg.block in (64, 128, 256)
    assert ms > 0
    a = M.het_loglike_batch_cfg(batch.refs, batch.offsets, th, "mixed", cfg).cpu().numpy()
    b = M.het_loglike_batch(batch.refs, batch.offsets, th, "mixed").cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def test_graph_replay(M, batch):
    """A captured batch replays to the same results; rewriting theta in place between
    replays (one sampler step per replay) gives the results of a direct launch."""
    import torch
    th = torch.from_numpy(batch.theta).cuda()
    out = torch.empty((3, th.shape[1]), dtype=torch.float64, device="cuda")
    cfg = M.het_config(4, 128, 1)
    graph = M.HetGraph(batch.refs, batch.offsets, th, out, "mixed", cfg)
    r1 = graph.launch().clone()
    direct = M.het_loglike_batch_cfg(batch.refs, batch.offsets, th, "mixed", cfg)
    torch.testing.assert_close(r1, direct, rtol=0, atol=0)
    th2 = th.clone()
    th2[I.I_MT] *= 1.0 + 1e-6
    th.copy_(th2)
    r2 = graph.launch().clone()
    direct2 = M.het_loglike_batch_cfg(batch.refs, batch.offsets, th2, "mixed", cfg)
    torch.testing.assert_close(r2, direct2, rtol=0, atol=0)
    assert not torch.equal(r1, r2)
    graph.close()


def test_bad_configuration_rejected(M, batch):
    import torch
    th = torch.from_numpy(batch.theta).cuda()
    with pytest.raises(M.MBHError):
        M.het_loglike_batch_cfg(batch.refs, batch.offsets, th, "mixed", M.het_config(3, 128, 0))
    for g, b in ((8, 100), (8, 288), (32, 224), (16, 160), (32, 16)):
        with pytest.raises(M.MBHError):
            M.het_loglike_batch_cfg(batch.refs, batch.offsets, th, "mixed", M.het_config(g, b, 0))
    with pytest.raises(M.MBHError):   # the float64 kernel has no 224-thread block
        M.het_loglike_batch_cfg(batch.refs, batch.offsets, th, "fp64", M.het_config(8, 224, 0))
