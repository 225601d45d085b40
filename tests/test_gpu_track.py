"""Feature tracking by projection on the GPU against the oracle: matched
index and best distance exact per query."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import compare_keypoints, frontend_for, params_from

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


def _run(J, oracle, frame, p, u, v, lv, desc, radius, max_dist=100):
    import torch
    fe = frontend_for(J, p)
    img = torch.from_numpy(frame).cuda()
    fe.extract(img, img, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    cu = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()
    idx, dist = fe.track(0, 0, cu(u, np.float32), cu(v, np.float32), cu(lv, np.uint8),
                         cu(np.asarray(desc, np.uint32).view(np.int32), np.int32), radius, max_dist)
    fe.sync()
    kf = oracle.extract_image(frame, p)
    compare_keypoints(J.to_numpy(fe.keypoints(0, 0)), kf, "frame")
    want_i, want_d = oracle.track(kf, p.scale, u, v, lv, desc, radius, max_dist)
    got_i = idx.cpu().numpy()
    got_d = dist.cpu().numpy().view(np.uint16)
    assert np.array_equal(got_i, want_i), np.nonzero(got_i != want_i)[0][:5]
    assert np.array_equal(got_d, want_d), np.nonzero(got_d != want_d)[0][:5]
    fe.close()
    return want_i, want_d


def test_track_self_and_translation(J, oracle):
    p = params_from(oracle, levels=6, max_feats=1500, fast_thresh_lo=7)
    a = scenes.workload_pair("kitti_1241x376_L8", 4).left
    ka = oracle.extract_image(a, p)
    n = ka["count"]
    u, v = ka["X"][:n].astype(np.float32), ka["Y"][:n].astype(np.float32)
    i, d = _run(J, oracle, a, p, u, v, ka["level"][:n], ka["desc"][:n], 0.5)
    assert (i == np.arange(n)).mean() > 0.95
    b = scenes.workload_pair("kitti_1241x376_L8", 5).left  # next frame (camera moved)
    i, d = _run(J, oracle, b, p, u + 0.5, v, ka["level"][:n], ka["desc"][:n], 8.0)
    assert (i >= 0).mean() > 0.3


def test_track_random_queries(J, oracle):
    p = params_from(oracle, levels=5, max_feats=1200, fast_thresh_lo=7)
    frame = scenes.planes_pair(640, 480, 0, 31, 32).left
    kf = oracle.extract_image(frame, p)
    rng = np.random.default_rng(9)
    n = 3000
    pick = rng.integers(0, kf["count"], n)
    u = kf["X"][pick].astype(np.float32) + rng.uniform(-6, 6, n).astype(np.float32)
    v = kf["Y"][pick].astype(np.float32) + rng.uniform(-6, 6, n).astype(np.float32)
    u[:50] = rng.uniform(-20, 0, 50)          # outside the image
    lv = kf["level"][pick].astype(np.uint8)
    lv[50:80] = rng.integers(5, 12, 30)        # beyond the frame's levels, some >= 8
    desc = kf["desc"][pick].copy()
    flip = rng.integers(0, 2, (n, 8)).astype(np.uint32) << rng.integers(0, 32, (n, 8)).astype(np.uint32)
    desc ^= flip                               # a few bits changed per word
    for radius, md in ((4.0, 100), (7.5, 40), (0.0, 256)):
        _run(J, oracle, frame, p, u, v, lv, desc, radius, md)


def test_track_errors(J, oracle):
    import torch
    p = params_from(oracle, levels=3, max_feats=300)
    fe = frontend_for(J, p)
    z = torch.zeros(4, dtype=torch.float32, device="cuda")
    lv = torch.zeros(4, dtype=torch.uint8, device="cuda")
    dsc = torch.zeros(4, 8, dtype=torch.int32, device="cuda")
    with pytest.raises(J.JslamError):
        fe.track(0, 0, z, z, lv, dsc, 3.0)      # before any extraction
    img = torch.from_numpy(scenes.planes_pair(320, 240, 0, 3, 4).left).cuda()
    fe.extract(img, img, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    for bad in (dict(radius=-1.0), dict(radius=3.0, max_dist=300)):
        with pytest.raises(J.JslamError):
            fe.track(0, 0, z, z, lv, dsc, **bad)
    with pytest.raises(J.JslamError):
        fe.track(3, 0, z, z, lv, dsc, 3.0)      # no such pair
    fe.close()
