"""Parity in the launch configuration the benchmark times: a 100-pair batch
(KITTI-shaped, EuRoC-shaped, 1920x1080) split over eight contexts on eight
streams, each part replayed as a captured CUDA graph, 128x128 detection
tiles.  Eight sampled pairs (one per context) are compared with the oracle
bit for bit; all 100 pairs are checked against properties that hold at any
size."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import compare_keypoints, compare_matches, params_from

pytestmark = pytest.mark.gpu

N = 100
PARTS = 8
SAMPLES = (0, 12, 25, 38, 50, 62, 75, 99)  # one per part (parts start at 0, 12, 25, 38, 50, 62, 75, 88)


@pytest.fixture(scope="module")
def J():
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


@pytest.fixture(scope="module", params=["kitti_1241x376_L8", "euroc_752x480_L8", "fhd_1920x1080_L8"])
def run(J, request):
    import torch
    WL = request.param
    w = scenes.WORKLOADS[WL]
    frames = [scenes.workload_pair(WL, f) for f in range(N)]
    dev = torch.device("cuda", 0)
    L = [torch.from_numpy(f.left).to(dev) for f in frames]
    R = [torch.from_numpy(f.right).to(dev) for f in frames]
    base = torch.cuda.current_stream()
    streams = [torch.cuda.Stream() for _ in range(PARTS)]
    bounds = [round(i * N / PARTS) for i in range(PARTS + 1)]
    fes = []
    for i in range(PARTS):
        sl = slice(bounds[i], bounds[i + 1])
        fe = J.Frontend(stream=streams[i], max_width=w["width"], max_height=w["height"], max_feats=w["max_feats"],
                        max_pairs=bounds[i + 1] - bounds[i], fast_thresh_lo=w["fast_thresh_lo"])
        fe.set_tuning(128, 128)
        jobs = fe.prepare_batch([J.Job(l, r, levels=w["levels"], scale=1.2, fast_thresh=w["fast_thresh"], cell=32,
                                       max_feats=w["max_feats"]) for l, r in zip(L[sl], R[sl])])
        fe.graph_capture(jobs)
        fes.append(fe)
    for _ in range(2):  # the second replay runs on buffers the first one used
        ev = torch.cuda.Event()
        ev.record(base)
        for s in streams:
            s.wait_event(ev)
        for fe in fes:
            fe.graph_launch()
        for fe in fes:
            fe.sync()
    out = []
    for i, fe in enumerate(fes):
        for p in range(bounds[i + 1] - bounds[i]):
            out.append((J.to_numpy(fe.keypoints(p, 0)), J.to_numpy(fe.keypoints(p, 1)), J.to_numpy(fe.matches(p))))
    yield frames, out, w
    for fe in fes:
        fe.close()


def test_sampled_pairs_match_the_oracle(J, oracle, run):
    frames, out, w = run
    p = params_from(oracle, levels=w["levels"], max_feats=w["max_feats"], fast_thresh=w["fast_thresh"],
                    fast_thresh_lo=w["fast_thresh_lo"])
    for k in SAMPLES:
        ol, orr, om = oracle.extract_pair(frames[k].left, frames[k].right, p)
        kl, kr, m = out[k]
        compare_keypoints(kl, ol, f"pair {k} left")
        compare_keypoints(kr, orr, f"pair {k} right")
        compare_matches(m, om, f"pair {k}")


def test_every_pair_is_well_formed(J, run):
    frames, out, w = run
    H0, W0 = frames[0].left.shape
    gw, gh, _ = J.level_geometry(W0, H0, w["levels"], 1.2, 32)
    for k, (kl, kr, m) in enumerate(out):
        for side, kp in ((0, kl), (1, kr)):
            n = kp["count"]
            assert 0 < n <= w["max_feats"], (k, side, n)
            lev, x, y = (np.asarray(kp[f][:n]).astype(np.int64) for f in ("level", "x", "y"))
            order = lev * (1 << 40) + y * (1 << 20) + x
            assert np.all(np.diff(order) > 0), (k, side)            # canonical (level, y, x), no repeats
            assert np.all(x >= 19) and np.all(y >= 19)
            assert np.all(x < gw[lev] - 19) and np.all(y < gh[lev] - 19)
            X, Y = np.asarray(kp["X"][:n]).astype(np.int64), np.asarray(kp["Y"][:n]).astype(np.int64)
            for i in range(0, n, 97):                                 # s0 projection of a spread of keypoints
                assert X[i] == J.project(int(x[i]), int(lev[i]), 1.2, W0)
                assert Y[i] == J.project(int(y[i]), int(lev[i]), 1.2, H0)
        n = kl["count"]
        idx = np.asarray(m["right_idx"][:n]).astype(np.int64)
        disp = np.asarray(m["disparity"][:n]).astype(np.int64)
        dist = np.asarray(m["dist"][:n]).astype(np.int64)
        ok = idx >= 0
        assert ok.sum() > n // 4, k
        XL, XR = np.asarray(kl["X"][:n]).astype(np.int64), np.asarray(kr["X"]).astype(np.int64)
        assert np.array_equal(disp[ok], XL[ok] - XR[idx[ok]])
        assert np.all((disp[ok] >= 0) & (disp[ok] <= 128)) and np.all(dist[ok] <= 100)
        lvl_l, lvl_r = np.asarray(kl["level"][:n]).astype(np.int64), np.asarray(kr["level"]).astype(np.int64)
        assert np.all(np.abs(lvl_l[ok] - lvl_r[idx[ok]]) <= 1)
