"""Failure detection without a GPU fault: a bounded device wait that runs
out is reported through the status codes, and forced allocation failures
(the JSLAM_FAIL_ALLOC_AFTER hook, host side) end in JSLAM_ERR_NOMEM with the
process and the device intact."""
import os
import subprocess
import sys
import time

import pytest

from paper_2410_04090_gb300 import scenes

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def J():
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


def _small_run(J):
    import torch
    pr = scenes.planes_pair(320, 240, 0, 5, 6)
    fe = J.Frontend(max_width=320, max_height=240, max_feats=300, max_pairs=1)
    fe.extract(torch.from_numpy(pr.left).cuda(), torch.from_numpy(pr.right).cuda(), levels=3, scale=1.2,
               fast_thresh=20, cell=32, max_feats=300)
    fe.match()
    fe.sync()
    n = fe.keypoints(0, 0)["count"]
    fe.close()
    return n


def test_bounded_wait_runs_out(J):
    fe = J.Frontend(max_width=320, max_height=240, max_feats=300, max_pairs=1)
    t0 = time.perf_counter()
    fe.selftest_wait()
    with pytest.raises(J.JslamError) as e:
        fe.sync()
    dt = time.perf_counter() - t0
    assert e.value.status == J.ERR_TIMEOUT
    assert 0.3 < dt < 20, dt          # the wait's limit is 2^31 SM cycles, about a second
    with pytest.raises(J.JslamError) as e2:
        fe.sync()                     # the context keeps its status
    assert e2.value.status == J.ERR_TIMEOUT
    fe.close()
    assert _small_run(J) > 0          # the device and a new context work


_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import torch
from paper_2410_04090_gb300 import jslam, scenes
pr = scenes.planes_pair(320, 240, 0, 5, 6)
try:
    fe = jslam.Frontend(max_width=320, max_height=240, max_feats=300, max_pairs=1)
    fe.extract(torch.from_numpy(pr.left).cuda(), torch.from_numpy(pr.right).cuda(), levels=3, scale=1.2,
               fast_thresh=20, cell=32, max_feats=300)
    fe.match()
    fe.sync()
    print("ok", fe.keypoints(0, 0)["count"])
    fe.close()
except jslam.JslamError as e:
    print("status", e.status)
"""


def test_forced_allocation_failures(J):
    """The (n+1)-th device allocation of the process fails: creation or the
    first extraction returns JSLAM_ERR_NOMEM; enough allowed allocations
    give the same keypoints as without the hook."""
    want = _small_run(J)
    seen = {}
    for n in (0, 1, 2, 3, 5, 8, 13, 1000):
        env = dict(os.environ, JSLAM_FAIL_ALLOC_AFTER=str(n))
        r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT)], env=env, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr[-2000:]
        out = r.stdout.strip().splitlines()[-1].split()
        seen[n] = out
        if out[0] == "status":
            assert int(out[1]) == J.ERR_NOMEM, (n, out)
        else:
            assert out[0] == "ok" and int(out[1]) == want, (n, out)
    assert seen[0][0] == "status"     # no allocation allowed: creation fails
    assert seen[1000][0] == "ok"      # no failure within the run
