"""Serving loop: continuous batching of heterodyne requests from concurrent samplers.
Failures are made on the host (cancelled requests, evicted sources, full queue,
exhausted budget, timeouts); nothing here faults or stalls the GPU."""
import threading
import time

import numpy as np
import pytest

import mbh_inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01064_b300 import mbhlike as M
    from paper_2111_01064_b300 import workloads as WL
    ub = WL.uneven_batch(n_sources=6, walkers=(16, 300))
    return M, WL, ub


def _req(ub, s, n=None, k=0):
    a, b = ub.offsets[s], ub.offsets[s + 1]
    th = ub.theta[:, a:b]
    if n is not None:
        th = th[:, k:k + n]
    return np.ascontiguousarray(th)


def test_request_same_alone_and_in_the_mix(env):
    """A request's results are bit-identical alone and packed with other samplers'
    requests (different sources, concurrent threads)."""
    M, WL, ub = env
    cfg = M.het_config(8, 128, 0)
    srv = M.Server(1 << 30, max_batch_walkers=4096, max_inflight_batches=3, cfg=cfg)
    ids = [srv.add_source(r) for r in ub.refs]
    probe = _req(ub, 2)
    st, alone = srv.wait(srv.submit(ids[2], probe))
    assert st == 0
    results, errors = {}, []

    def sampler(s):
        try:
            for rep in range(5):
                rid = srv.submit(ids[s], _req(ub, s))
                results[(s, rep)] = srv.wait(rid)
        except Exception as exc:   # pragma: no cover
            errors.append(exc)

    threads = [threading.Thread(target=sampler, args=(s,)) for s in range(len(ids))]
    for t in threads:
        t.start()
    mixed = [srv.submit(ids[2], probe) for _ in range(3)]
    for t in threads:
        t.join()
    assert not errors
    for rid in mixed:
        st, out = srv.wait(rid)
        assert st == 0
        np.testing.assert_array_equal(out, alone)
    # and the same as a direct launch with the same configuration
    import torch
    direct = M.het_loglike_batch_cfg([ub.refs[2]], [0, probe.shape[1]], torch.from_numpy(probe).cuda(),
                                     "mixed", cfg).cpu().numpy()
    np.testing.assert_array_equal(alone, direct)
    for (s, rep), (st, out) in results.items():
        assert st == 0 and np.all(np.isfinite(out))
    rep = srv.stats()
    assert rep["completed"] == 4 + 5 * len(ids) - 0 and rep["batches"] >= 1
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    srv.close()


def test_admission_by_memory_budget(env):
    """Slots and resident sources are admitted only while they fit the budget."""
    M, WL, ub = env
    with pytest.raises(M.MBHError) as e:
        M.Server(1 << 10, max_batch_walkers=4096, max_inflight_batches=2)
    assert e.value.status == 5
    probe = M.Server(1 << 30, max_batch_walkers=256, max_inflight_batches=2)
    probe.add_source(ub.refs[0])
    rep = probe.stats()
    probe.close()
    srv = M.Server(rep["slot_bytes"] + rep["source_bytes"] + 16, max_batch_walkers=256,
                   max_inflight_batches=2)
    srv.add_source(ub.refs[0])
    with pytest.raises(M.MBHError) as e:
        srv.add_source(ub.refs[0])          # a second copy no longer fits
    assert e.value.status == 5
    assert srv.stats()["rejected"] == 1
    srv.close()


def test_queue_full_cancel_timeout_and_eviction(env):
    M, WL, ub = env
    srv = M.Server(1 << 30, max_batch_walkers=4096, max_inflight_batches=2, max_queue=4)
    a, b = srv.add_source(ub.refs[0]), srv.add_source(ub.refs[1])
    srv.pause(True)
    r1 = srv.submit(a, _req(ub, 0, 8))
    r2 = srv.submit(b, _req(ub, 1, 8))
    r3 = srv.submit(a, _req(ub, 0, 8, 8))
    r4 = srv.submit(b, _req(ub, 1, 8, 8))
    with pytest.raises(M.MBHError) as e:
        srv.submit(a, _req(ub, 0, 8))
    assert e.value.status == 5                      # queue full
    with pytest.raises(M.MBHError) as e:
        srv.wait(r1, timeout_ms=50)
    assert e.value.status == 4                      # timed out (paused)
    srv.cancel(r3)
    st, _ = srv.wait(r3, 0)
    assert st == 6                                   # cancelled
    srv.remove_source(b)                            # evict while r2, r4 are queued
    assert srv.wait(r2, 0)[0] == 1 and srv.wait(r4, 0)[0] == 1
    srv.pause(False)
    st, out = srv.wait(r1, timeout_ms=10_000)
    assert st == 0 and np.all(np.isfinite(out))
    with pytest.raises(M.MBHError):
        srv.submit(b, _req(ub, 1, 8))               # unknown (evicted) source
    with pytest.raises(M.MBHError):
        srv.cancel(r1)                               # already done and collected
    srv.close()


def test_slow_producer_and_shutdown(env):
    M, WL, ub = env
    srv = M.Server(1 << 30, max_batch_walkers=1024, max_inflight_batches=2)
    sid = srv.add_source(ub.refs[3])
    outs = []
    for k in range(4):
        outs.append(srv.submit(sid, _req(ub, 3, 4, 4 * k)))
        time.sleep(0.02)
    for rid in outs:
        assert srv.wait(rid, timeout_ms=10_000)[0] == 0
    srv.pause(True)
    pending = srv.submit(sid, _req(ub, 3, 4))
    srv.close()                                      # cancels what was never launched


def test_reference_refresh_hot_swap(env):
    """Reference refresh: re-prepare around the best walker of a batch (band re-selected)
    and swap it into the running server; later requests use the new reference and give
    the results of a direct launch with it."""
    import torch
    M, WL, ub = env
    cfg = M.het_config(8, 128, 0)
    src = ub.sources[4]
    srv = M.Server(1 << 30, max_batch_walkers=4096, max_inflight_batches=2, cfg=cfg)
    sid = srv.add_source(ub.refs[4])
    th = _req(ub, 4)
    st, out = srv.wait(srv.submit(sid, th))
    assert st == 0
    best = int(np.argmax(out[0]))
    new_ref = M.het_prepare_reference(src.data, th[:, best], int(ub.bins[4]))
    pending = [srv.submit(sid, th) for _ in range(3)]
    srv.replace_source(sid, new_ref)
    after = srv.submit(sid, th)
    direct_new = M.het_loglike_batch_cfg([new_ref], [0, th.shape[1]], torch.from_numpy(th).cuda(),
                                         "mixed", cfg).cpu().numpy()
    st, got = srv.wait(after)
    assert st == 0
    np.testing.assert_array_equal(got, direct_new)
    # requests submitted before the swap were evaluated with one of the two references
    direct_old = M.het_loglike_batch_cfg([ub.refs[4]], [0, th.shape[1]], torch.from_numpy(th).cuda(),
                                         "mixed", cfg).cpu().numpy()
    for rid in pending:
        st, o = srv.wait(rid)
        assert st == 0
        assert np.array_equal(o, direct_old) or np.array_equal(o, direct_new)
    # at the new reference (r = 1) the heterodyne equals the direct lnL to the mixed bound
    dr = M.direct_loglike_batch(src.data, torch.from_numpy(th).cuda(), "fp64").cpu().numpy()
    assert abs(got[0, best] - dr[0, best]) <= 1e-3
    srv.close()


def test_native_load_generator(env):
    """Client threads in the library drive the server at Poisson arrival times: every accepted
    request completes, the latency statistics cover them, and invalid options are refused."""
    M, WL, ub = env
    srv = M.Server(1 << 30, max_batch_walkers=16384, max_inflight_batches=3, precision="mixed")
    ids = [srv.add_source(r) for r in ub.refs[:4]]
    P = int(min(ub.offsets[s + 1] - ub.offsets[s] for s in range(4)))
    pools = [np.ascontiguousarray(ub.theta[:, ub.offsets[s]:ub.offsets[s] + P]) for s in range(4)]
    rep = srv.loadgen(ids, pools, 400.0, 0.5, 1, P, seed=3)
    assert rep["submitted"] > 100 and rep["completed"] == rep["submitted"] and rep["failed"] == 0
    assert 0 < rep["p50_ms"] <= rep["p99_ms"] <= rep["max_ms"]
    assert srv.stats()["completed"] == rep["completed"]
    with pytest.raises(M.MBHError):
        srv.loadgen(ids, pools, 400.0, 0.5, 1, P + 1)    # larger than the pools
    with pytest.raises(M.MBHError):
        srv.loadgen(ids, pools, 0.0, 0.5, 1, P)
    srv.close()
