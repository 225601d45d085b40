"""Parity of the two off-by-default readings with the oracle, through the C
ABI: the arc response (response_mode = 1; Sec. III's response read as the
sum of (|d| - eps) over the qualifying arc) in the bit-sliced detection
kernel, the table kernel for other run bounds, and the ablation's
CRF-matrix; the cascaded pyramid (pyramid_mode = 1; level n resampled from
level n - 1), its levels byte for byte, and a captured graph of it replayed
on new frames.  Bit-exact keypoints, scores, sectors, descriptors and
matches; angles within 1e-4 rad."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import compare_keypoints, compare_matches, frontend_for, gpu_pair, params_from

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


def _check(J, oracle, pair, p, **fe_kw):
    fe = frontend_for(J, p, **fe_kw)
    try:
        kl, kr, m = gpu_pair(J, fe, pair.left, pair.right, p)
    finally:
        fe.close()
    ol, orr, om = oracle.extract_pair(pair.left, pair.right, p)
    compare_keypoints(kl, ol, "left")
    compare_keypoints(kr, orr, "right")
    compare_matches(m, om, "matches")
    return ol


@pytest.mark.parametrize("workload,p_min,p_max,lo", [
    ("kitti_1241x376_L8", 9, 13, 7),     # bit-sliced kernel, fallback corners ranked at eps_lo
    ("euroc_752x480_L8", 9, 13, 7),      # many fallback cells
    ("kitti_1241x376_L8", 9, 16, 7),     # table kernel (other run bounds)
    ("euroc_752x480_L8", 8, 12, 0),      # table kernel, both polarities may qualify, no fallback
])
def test_arc_response_parity(J, oracle, workload, p_min, p_max, lo):
    pair = scenes.workload_pair(workload, 3)
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=lo, p_min=p_min, p_max=p_max, response_mode=1)
    ol = _check(J, oracle, pair, p)
    assert ol["count"] > 500
    # the arc reading ranks differently from the default one on this pair
    q = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=lo, p_min=p_min, p_max=p_max)
    od = oracle.extract_image(pair.left, q)
    assert not (od["count"] == ol["count"] and np.array_equal(od["response"], ol["response"]))


def test_arc_response_crf_matrix(J, oracle):
    """The ablation's CRF-matrix in arc mode: every level equals the oracle's
    arc CRF at the primary threshold, and its per-cell keys equal the fused
    kernel's (fallback off)."""
    import torch
    pair = scenes.workload_pair("kitti_1241x376_L8", 1)
    p = params_from(oracle, levels=4, max_feats=4000, response_mode=1)
    fe = frontend_for(J, p)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(), p.levels, p.scale,
               p.fast_thresh, p.cell, p.max_feats)
    fe.fc_ablation(8)
    fe.sync()
    H0, W0 = pair.left.shape
    for n in range(p.levels):
        lvl = pair.left if n == 0 else oracle.pyramid_level(pair.left, p.scale, n)
        _, want = oracle.fast_arc(lvl, p.fast_thresh, p.p_min, p.p_max, p.border)
        got = fe.crf(0, 0, n).cpu().numpy()
        assert np.array_equal(got, want), n
        abl, fused = fe.fc_ablation_keys(0, 0, n)
        assert np.array_equal(abl.cpu().numpy(), fused.cpu().numpy()), n
    fe.close()


def test_cascaded_pyramid_parity(J, oracle):
    import torch
    pair = scenes.workload_pair("kitti_1241x376_L8", 2)
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=7, pyramid_mode=1)
    _check(J, oracle, pair, p)
    # the raw levels themselves: level n resampled from level n - 1
    fe = frontend_for(J, p)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(), p.levels, p.scale,
               p.fast_thresh, p.cell, p.max_feats)
    fe.sync()
    W, H, _ = oracle.level_geometry(pair.left.shape[1], pair.left.shape[0], p.levels, p.scale, p.cell)
    prev = pair.right
    direct_differs = False
    for n in range(1, p.levels):
        want = oracle.pyramid_level_sized(prev, p.scale, 1, int(W[n]), int(H[n]))
        got = fe.level(0, 1, n)["raw"].cpu().numpy()
        assert np.array_equal(got, want), n
        direct_differs |= not np.array_equal(want, oracle.pyramid_level(pair.right, p.scale, n))
        prev = want
    assert direct_differs
    fe.close()


def test_cascaded_pyramid_graph_on_new_frames(J, oracle):
    """A captured graph of the cascaded pyramid (one pyramid launch per
    level) replayed on new device frames."""
    import torch
    p = params_from(oracle, levels=6, max_feats=2000, fast_thresh_lo=7, pyramid_mode=1, response_mode=1)
    fe = frontend_for(J, p, max_pairs=2, stream=torch.cuda.Stream())
    mk = lambda f: [scenes.workload_pair("euroc_752x480_L8", f + i) for i in range(2)]
    jobs = lambda prs: [J.Job(torch.from_numpy(pr.left).cuda(), torch.from_numpy(pr.right).cuda(), p.levels, p.scale,
                              p.fast_thresh, p.cell, p.max_feats) for pr in prs]
    j0 = jobs(mk(0))
    torch.cuda.synchronize()
    fe.graph_capture(j0)
    new = mk(10)
    j1 = jobs(new)
    torch.cuda.synchronize()
    fe.graph_launch(j1)
    fe.sync()
    for i, pr in enumerate(new):
        ol, orr, om = oracle.extract_pair(pr.left, pr.right, p)
        compare_keypoints(J.to_numpy(fe.keypoints(i, 0)), ol, f"pair {i} left")
        compare_keypoints(J.to_numpy(fe.keypoints(i, 1)), orr, f"pair {i} right")
        compare_matches(J.to_numpy(fe.matches(i)), om, f"pair {i}")
    fe.close()
