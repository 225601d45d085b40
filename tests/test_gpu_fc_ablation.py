"""The paper-style feature culling (CRF-matrix + MLPT/TEWA kernels) kept as
an ablation baseline: its per-cell keys equal the fused detection kernel's
and the oracle's culling (Sec. II-C-1) at the primary threshold."""
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


def _oracle_keys(oracle, img0, p, n):
    W0 = img0.shape[1]; H0 = img0.shape[0]
    w, h, c = oracle.level_geometry(W0, H0, p.levels, p.scale, p.cell)
    Wn, Hn, cn = int(w[n]), int(h[n]), int(c[n])
    lev = img0 if n == 0 else oracle.pyramid_level_sized(img0, p.scale, n, Wn, Hn)
    corner, resp = oracle.fast(lev, p.fast_thresh, p.p_min, p.p_max, p.border)
    xs, ys, rs = oracle.cull_level(corner, None, resp, cn, 1)
    keys = np.zeros(((Hn + cn - 1) // cn, (Wn + cn - 1) // cn), np.uint32)
    for x, y, r in zip(xs, ys, rs):
        cx, cy = x // cn, y // cn
        keys[cy, cx] = (int(r) << 16) | (0xFFFF - ((y - cy * cn) * cn + (x - cx * cn)))
    return keys


def test_ablation_matches_fused_and_oracle(J, oracle):
    import torch
    pair = scenes.workload_pair("kitti_1241x376_L8", 6)
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=0)
    fe = frontend_for(J, p)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(), p.levels, p.scale,
               p.fast_thresh, p.cell, p.max_feats)
    want = {(s, n): _oracle_keys(oracle, img, p, n) for s, img in enumerate((pair.left, pair.right))
            for n in range(p.levels)}
    for n_max in (8, 4, 16):
        fe.fc_ablation(n_max)
        fe.sync()
        for (s, n), w in want.items():
            a, f = fe.fc_ablation_keys(0, s, n)
            a, f = a.cpu().numpy(), f.cpu().numpy()
            assert np.array_equal(f, w), (s, n)
            assert np.array_equal(a, w), (n_max, s, n, np.argwhere(a != w)[:3])
    t = fe.fc_ablation_times()
    assert t["crf_ms"] > 0 and t["fc_ms"] > 0
    fe.close()


def test_ablation_arguments(J, oracle):
    import torch
    p = params_from(oracle, levels=3, max_feats=300)
    fe = frontend_for(J, p)
    with pytest.raises(J.JslamError):
        fe.fc_ablation(8)                      # before an extraction
    img = torch.from_numpy(scenes.planes_pair(320, 240, 0, 3, 4).left).cuda()
    fe.extract(img, img, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    with pytest.raises(J.JslamError):
        fe.fc_ablation(1)                      # 32-pixel cells would need 32 x 128 threads
    fe.close()
    p3 = params_from(oracle, levels=3, max_feats=300, k_per_cell=3)
    fe = frontend_for(J, p3)
    fe.extract(img, img, p3.levels, p3.scale, p3.fast_thresh, p3.cell, p3.max_feats)
    with pytest.raises(J.JslamError):
        fe.fc_ablation(8)                      # the paper's culling keeps one corner per cell
    fe.close()
