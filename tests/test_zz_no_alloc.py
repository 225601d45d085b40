"""The allocation-free entry point jslam_pfa_scores_static, for callers that
cannot allocate device memory (real-time loops that forbid allocation after
start-up, plug-ins inside another framework's enqueue hook, fixed memory
pools), gives the same PFA scores as the full extraction (jslam_extract):
the same surviving corners and, for each, the same s0 projection, K_l and
K_r.  Two calls in a row on different images check that the shared static
scratch table is cleared between calls.  This file is collected last."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import frontend_for, params_from

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


def _culled_corners(oracle, img, p):
    """Per-cell culled corners of every level of `img`: (level, x, y, response)."""
    H0, W0 = img.shape
    _, _, cells = oracle.level_geometry(W0, H0, p.levels, p.scale, p.cell)
    cols = [[], [], [], []]
    for n in range(p.levels):
        lvl = img if n == 0 else oracle.pyramid_level(img, p.scale, n)
        hi, resp = oracle.fast(lvl, p.fast_thresh, p.p_min, p.p_max, p.border)
        lo = oracle.fast(lvl, p.fast_thresh_lo, p.p_min, p.p_max, p.border)[0] if p.fast_thresh_lo > 0 else None
        xs, ys, rs = oracle.cull_level(hi, lo, resp, int(cells[n]), p.k_per_cell)
        cols[0] += [n] * len(xs); cols[1] += xs.tolist(); cols[2] += ys.tolist(); cols[3] += rs.tolist()
    return (np.array(cols[0], np.uint8), np.array(cols[1], np.uint16), np.array(cols[2], np.uint16),
            np.array(cols[3], np.uint16))


def test_static_scratch_pfa_matches_extract(J, oracle):
    import torch
    pair = scenes.workload_pair("kitti_1241x376_L8", 5)
    p = params_from(oracle, levels=8, max_feats=8000, fast_thresh_lo=7)  # no cap: every survivor is kept
    fe = frontend_for(J, p, max_feats=8000)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(),
               p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.sync()
    H0, W0 = pair.left.shape
    for side, img in ((0, pair.left), (1, pair.right)):  # two calls in a row
        kp = J.to_numpy(fe.keypoints(0, side))
        lv, xs, ys, rs = _culled_corners(oracle, img, p)
        assert len(lv) > kp["count"] > 500
        t = [torch.from_numpy(a).cuda() for a in (lv, xs, ys, rs)]
        out = J.pfa_scores_static(*t, width0=W0, height0=H0, levels=p.levels, scale=p.scale,
                                  nms_q=p.nms_q, pfa_rule=p.pfa_rule)
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy() for k, v in out.items()}
        keep = out["alive"].astype(bool)
        got = sorted(zip(lv[keep].tolist(), ys[keep].tolist(), xs[keep].tolist(), out["X"][keep].tolist(),
                         out["Y"][keep].tolist(), out["k_levels"][keep].tolist(), out["k_resp"][keep].tolist(),
                         rs[keep].tolist()))
        want = sorted(zip(kp["level"].tolist(), kp["y"].tolist(), kp["x"].tolist(), kp["X"].tolist(),
                          kp["Y"].tolist(), kp["k_levels"].tolist(), kp["k_resp"].tolist(),
                          kp["response"].tolist()))
        assert got == want, f"side {side}"
    fe.close()


def test_static_scratch_rejects_oversize(J):
    import torch
    n = 16385
    z8 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    z16 = torch.zeros(n, dtype=torch.uint16, device="cuda")
    with pytest.raises(J.JslamError) as e:
        J.pfa_scores_static(z8, z16, z16, z16, width0=640, height0=480, levels=1)
    assert e.value.status == J.ERR_CAPACITY
    with pytest.raises(J.JslamError) as e:
        J.pfa_scores_static(z8[:10], z16[:10], z16[:10], z16[:10], width0=640, height0=480, levels=1, nms_q=2)
    assert e.value.status == J.ERR_ARG
