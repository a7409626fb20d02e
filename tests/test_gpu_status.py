"""Device-side status word (mbh_sync_status) and the in-kernel index checks of the debug build.

Release build: no in-kernel checks; mbh_sync_status synchronises and reports nothing after
normal work, and the debug hook is refused.  Debug build (libmbhlike_debug.so, loaded in a
child process with MBH_DEBUG_CHECKS=1): the reference's logical edge range is narrowed to
[0, E/2] with mbh_debug_ref_limit, so the heterodyne kernels meet edge indices past it that
are still inside the allocated edge records (the kernels' loops and tables are unchanged):
each kernel records the first such index in the status word, skips the access and returns;
mbh_sync_status reports it once (MBH_EDEVICE) and clears it, and with the range restored the
results are bit-identical to a run that never tripped.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import mbh_inputs as I

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MBH_EDEVICE = 7


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_01064_b300 import mbhlike
    mbhlike.lib()
    return mbhlike


def test_sync_status_release_build(M):
    from paper_2111_01064_b300 import workloads as WL
    assert not M.mbh_debug_checks()
    g = I.grid_month()
    src = WL.source_for(0, g)
    ref = M.het_prepare_reference(src.data, src.theta_inj, 32)
    th = WL.to_dev(WL.walkers(src.theta_inj, 16, 0, lo=1e-5, hi=1e-3))
    for prec in ("mixed", "mixed_f32", "fp64"):
        M.het_loglike_batch([ref], [0, 16], th, prec)
        st, info = M.mbh_sync_status()
        assert st == 0 and info["code"] == 0
    with pytest.raises(M.MBHError) as e:
        M.mbh_debug_ref_limit(ref, 4)
    assert e.value.status == 1


CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import mbh_inputs as I
from paper_2111_01064_b300 import mbhlike as M, workloads as WL
assert M.mbh_debug_checks()
g = I.grid_month()
src = WL.source_for(0, g)
ref = M.het_prepare_reference(src.data, src.theta_inj, 64)
E = ref.bins
W = 32
th = WL.to_dev(WL.walkers(src.theta_inj, W, 0, lo=1e-5, hi=1e-3))
res = {"E": E}
for prec in ("mixed", "mixed_f32", "fp64"):
    base = M.het_loglike_batch([ref], [0, W], th, prec).cpu().numpy()
    st0, _ = M.mbh_sync_status()
    M.mbh_debug_ref_limit(ref, E // 2)
    M.het_loglike_batch([ref], [0, W], th, prec)
    st1, info = M.mbh_sync_status()
    st2, _ = M.mbh_sync_status()
    M.mbh_debug_ref_limit(ref, -1)
    again = M.het_loglike_batch([ref], [0, W], th, prec).cpu().numpy()
    st3, _ = M.mbh_sync_status()
    res[prec] = dict(st0=st0, st1=st1, info=info, st2=st2, st3=st3, same=bool(np.array_equal(base, again)))
print("RESULT " + json.dumps(res))
"""


def test_debug_build_records_and_skips_out_of_range_edges(M):
    from paper_2111_01064_b300 import build
    build.build(debug=True)
    env = dict(os.environ, MBH_DEBUG_CHECKS="1")
    p = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    line = [ln for ln in p.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    E = res["E"]
    for prec, kernel in (("mixed", 1), ("mixed_f32", 2), ("fp64", 3)):
        r = res[prec]
        info = r["info"]
        assert r["st0"] == 0, prec
        assert r["st1"] == MBH_EDEVICE, prec
        assert info["code"] == 1 and info["kernel"] == kernel and info["source"] == 0, (prec, info)
        assert info["limit"] == E // 2 + 1 and E // 2 < info["index"] <= E, (prec, info)
        assert r["st2"] == 0 and r["st3"] == 0, prec
        assert r["same"], prec
