"""Correlation minimisation (sub-pixel stereo refinement) on the GPU against
the oracle: per left keypoint the SAD and every accept/reject decision are
exact; disparity and depth, computed in float on the GPU from the same
integers the oracle turns into doubles, agree within float rounding."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import compare_keypoints, compare_matches, frontend_for, params_from
from test_oracle_subpixel import smooth_texture

pytestmark = pytest.mark.gpu

BF = float(np.float32(386.1448))  # fx * baseline of a KITTI-like rig, exact in float


@pytest.fixture(scope="module")
def J():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


def _compare(got, want, what):
    """Tolerance from the float path: delta = num / den, one subtraction and
    one multiply by zeta^n (<= 3.6 at level 7), each rounded once: the
    disparity is within 2e-6 max(1, d) of the double value, the depth within
    the same relative error scaled by 1 / max(d, 0.01) plus one division."""
    n = len(want["disparity"])
    assert got["count"] == n, what
    g_sad, w_sad = np.asarray(got["sad"])[:n], np.asarray(want["sad"])
    assert np.array_equal(g_sad, w_sad), f"{what}: SAD differs at {np.nonzero(g_sad != w_sad)[0][:5]}"
    gd = np.asarray(got["disparity"])[:n].astype(np.float64)
    wd = np.asarray(want["disparity"]).astype(np.float64)
    keep = wd >= 0
    assert np.array_equal(gd >= 0, keep), f"{what}: accept/reject differs at {np.nonzero((gd >= 0) != keep)[0][:5]}"
    assert (gd[~keep] == -1).all()
    tol_d = 2e-6 * np.maximum(1.0, wd)
    assert (np.abs(gd - wd)[keep] <= tol_d[keep]).all(), f"{what}: disparity {np.abs(gd - wd)[keep].max()}"
    gz = np.asarray(got["depth"])[:n].astype(np.float64)
    wz = np.asarray(want["depth"]).astype(np.float64)
    tol_z = wz * (tol_d / np.maximum(wd, 0.01) + 1e-6)
    assert (np.abs(gz - wz) <= tol_z).all() and (gz[~keep] == 0).all(), f"{what}: depth"


def _pair(J, oracle, left, right, p, w=5, L=5, bf=BF):
    import torch
    fe = frontend_for(J, p)
    fe.extract(torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), p.levels, p.scale, p.fast_thresh,
               p.cell, p.max_feats)
    fe.match()
    fe.refine_matches(w, L, bf)
    fe.sync()
    kl, kr, m = oracle.extract_pair(left, right, p)
    compare_keypoints(J.to_numpy(fe.keypoints(0, 0)), kl, "left")
    compare_matches(J.to_numpy(fe.matches(0)), m)
    want = oracle.subpixel(left, right, kl, kr, m[0], p, w, L, bf)
    got = J.to_numpy(fe.refined(0))
    _compare(got, want, "pair")
    fe.close()
    return want


@pytest.mark.parametrize("name", ["kitti_1241x376_L8", "euroc_752x480_L8"])
def test_refine_workload_parity(J, oracle, name):
    w = scenes.WORKLOADS[name]
    pair = scenes.workload_pair(name, 9)
    p = params_from(oracle, levels=8, max_feats=w["max_feats"], fast_thresh_lo=w["fast_thresh_lo"])
    want = _pair(J, oracle, pair.left, pair.right, p)
    assert (want["disparity"] >= 0).sum() > 100


def test_refine_fractional_scene_and_variants(J, oracle):
    left = smooth_texture(300, 420, 0.0, 11)
    right = smooth_texture(300, 420, 10.25, 11)
    p = params_from(oracle, levels=4, max_feats=1500, fast_thresh=15, max_disp=64, match_max_dist=80)
    want = _pair(J, oracle, left, right, p)
    ok = want["disparity"] >= 0
    assert np.median(np.abs(want["disparity"][ok] - 10.25)) < 0.15
    _pair(J, oracle, left, right, p, w=3, L=7, bf=0.0)
    _pair(J, oracle, left, right, p, w=10, L=1, bf=BF)


def test_refine_batch_and_download(J, oracle):
    import torch
    p = params_from(oracle, levels=5, max_feats=700, fast_thresh_lo=7)
    prs = [scenes.planes_pair(420, 300, 0, 60 + k, 70 + k) for k in range(2)] + [scenes.planes_pair(300, 200, 0, 80, 81)]
    fe = frontend_for(J, p, max_pairs=4)
    jobs = [J.Job(torch.from_numpy(pr.left).cuda(), torch.from_numpy(pr.right).cuda(), p.levels, p.scale,
                  p.fast_thresh, p.cell, p.max_feats) for pr in prs]
    fe.extract_batch(jobs)
    fe.match()
    fe.refine_matches(5, 5, BF)
    total, offs = fe.result_range(0, 3)
    blk = torch.empty(total, dtype=torch.uint8).pin_memory()
    fe.download_range(0, 3, blk)
    fe.sync()
    for k, pr in enumerate(prs):
        kl, kr, m = oracle.extract_pair(pr.left, pr.right, p)
        want = oracle.subpixel(pr.left, pr.right, kl, kr, m[0], p, 5, 5, BF)
        _compare(J.to_numpy(fe.refined(k)), want, f"pair {k}")
        _compare(fe.result_refined_view(k, blk[offs[k]:].clone()), want, f"pair {k} block")
    fe.close()


def test_refine_errors_and_timing(J, oracle):
    import torch
    p = params_from(oracle, levels=3, max_feats=400)
    pair = scenes.planes_pair(320, 240, 0, 5, 6)
    fe = frontend_for(J, p)
    l, r = torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda()
    fe.extract(l, r, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    with pytest.raises(J.JslamError):
        fe.refine_matches(5, 5, 0.0)          # before jslam_match
    fe.match()
    for bad in ((0, 5, 0.0), (11, 5, 0.0), (5, 0, 0.0), (5, 8, 0.0), (5, 5, -1.0)):
        with pytest.raises(J.JslamError):
            fe.refine_matches(*bad)
    fe.enable_stage_timing(True)
    fe.extract(l, r, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    fe.refine_matches(5, 5, BF)
    fe.sync()
    t = fe.stage_times()
    assert t["refine"] > 0 and t["match"] > 0
    fe.close()
