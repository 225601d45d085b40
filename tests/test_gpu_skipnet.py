"""The learned cell-skip proposal: its inference kernel against a plain
PyTorch fp32 reference of the same net, the exact path when nothing is
skipped, and the feature recall of the trained model against the exact
path on held-out frames."""
import json
import os
import struct

import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import compare_keypoints, compare_matches, frontend_for, params_from

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
MODEL = os.path.join(os.path.dirname(HERE), "paper_2410_04090_gb300", "skipnet_v1.bin")


@pytest.fixture(scope="module")
def J():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


def _random_blob(seed=0):
    import torch
    from paper_2410_04090_gb300 import skipnet_train as T
    torch.manual_seed(seed)
    model = T.build_model(torch)
    T.round_weights_bf16(torch, model)
    return T.export_blob(torch, model), model


def _reference_logits(model, img):
    """fp64 convolutions with the kernel's rounding points (input and
    activations rounded to BF16)."""
    import torch
    from paper_2410_04090_gb300 import skipnet_train as T
    x = torch.from_numpy(T.box_mean(img))[None, None].double()
    with torch.no_grad():
        return T.forward_bf16(torch, model.double(), x)[0, 0].numpy()


def test_blob_layout(J):
    blob, _ = _random_blob()
    assert blob[:4] == b"JSKP" and struct.unpack("<III", blob[4:16]) == (1, 16, 8)
    fe = J.Frontend(device=0, max_width=320, max_height=240, max_pairs=1)
    with pytest.raises(J.JslamError):
        fe.set_skip_model(blob[:-2], 0.0)
    with pytest.raises(J.JslamError):
        fe.set_skip_model(b"XXXX" + blob[4:], 0.0)
    fe.set_skip_model(blob, 0.0)
    fe.set_skip_model(None)
    fe.close()


def test_skipnet_logits_match_torch(J, oracle):
    import torch
    blob, model = _random_blob(3)
    pair = scenes.planes_pair(437, 301, 0, 21, 22)  # ragged 1/8 map: 55 x 38
    p = params_from(oracle, levels=3, max_feats=600)
    fe = frontend_for(J, p)
    fe.set_skip_model(blob, 0.0)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(), p.levels, p.scale,
               p.fast_thresh, p.cell, p.max_feats)
    fe.sync()
    for side, img in ((0, pair.left), (1, pair.right)):
        v = fe.skip_view(0, side)
        got = v["logits"].cpu().numpy().astype(np.float64)
        want = _reference_logits(model, img)
        assert got.shape == want.shape == (38, 55)
        # FP32 tensor-core accumulation vs fp64: an activation that sits on a
        # BF16 rounding boundary may round the other way (one BF16 ulp, 2^-8
        # relative), so a few logits move by ~1e-3; most agree to ~1e-6.
        scale = max(1.0, np.abs(want).max())
        err = np.abs(got - want)
        assert err.max() <= 1e-2 * scale, err.max()
        assert np.median(err) <= 1e-5 * scale, np.median(err)
        # a cell is skipped when its largest logit is below the threshold
        cy, cx = v["skip"].shape
        cells = np.full((cy, cx), -np.inf)
        for y in range(got.shape[0]):
            for x in range(got.shape[1]):
                cells[(8 * y) // 32, (8 * x) // 32] = max(cells[(8 * y) // 32, (8 * x) // 32], got[y, x])
        assert np.array_equal(v["skip"].cpu().numpy().astype(bool), cells < 0.0)
    fe.close()


def test_nothing_skipped_is_exact(J, oracle):
    import torch
    blob, _ = _random_blob(5)
    pair = scenes.workload_pair("kitti_1241x376_L8", 7)
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=7)
    fe = frontend_for(J, p)
    fe.set_skip_model(blob, -1e30)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(), p.levels, p.scale,
               p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    fe.sync()
    ol, orr, om = oracle.extract_pair(pair.left, pair.right, p)
    compare_keypoints(J.to_numpy(fe.keypoints(0, 0)), ol, "left")
    compare_keypoints(J.to_numpy(fe.keypoints(0, 1)), orr, "right")
    compare_matches(J.to_numpy(fe.matches(0)), om)
    fe.close()


def test_everything_skipped(J, oracle):
    import torch
    blob, _ = _random_blob(6)
    pair = scenes.planes_pair(400, 300, 0, 1, 2)
    p = params_from(oracle, levels=4, max_feats=500)
    fe = frontend_for(J, p)
    fe.set_skip_model(blob, 1e30)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(), p.levels, p.scale,
               p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    fe.sync()
    assert fe.keypoints(0, 0)["count"] == 0 and fe.keypoints(0, 1)["count"] == 0
    fe.set_skip_model(None)  # back to the exact path
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(), p.levels, p.scale,
               p.fast_thresh, p.cell, p.max_feats)
    fe.sync()
    compare_keypoints(J.to_numpy(fe.keypoints(0, 0)), oracle.extract_image(pair.left, p), "left")
    fe.close()


@pytest.mark.skipif(not os.path.exists(MODEL), reason="trained skip model not present")
@pytest.mark.parametrize("kind,w,h,feats", [("planes", 1920, 1080, 3000), ("euroc", 752, 480, 1200)])
def test_trained_model_recall(J, oracle, kind, w, h, feats):
    """Feature recall of the trained proposal on held-out frames (scene seeds
    never seen in training) against the exact path: >= 99 %."""
    import torch
    meta = json.load(open(os.path.splitext(MODEL)[0] + ".json"))
    blob = open(MODEL, "rb").read()
    p = params_from(oracle, levels=8, max_feats=feats, fast_thresh_lo=7)
    exact = frontend_for(J, p)
    skip = frontend_for(J, p)
    skip.set_skip_model(blob, meta["thresh"])
    inter = total = kept = 0
    skipped = []
    for k in range(4):
        pr = scenes.stereo_pair(kind, w, h, frame=k, stream=200000 + k, config_id=5)
        l = torch.from_numpy(pr.left).cuda(); r = torch.from_numpy(pr.right).cuda()
        for fe in (exact, skip):
            fe.extract(l, r, 8, 1.2, 20, 32, feats)
            fe.sync()
        skipped.append(float(skip.skip_view(0, 0)["skip"].float().mean()))
        for side in (0, 1):
            a = J.to_numpy(exact.keypoints(0, side)); b = J.to_numpy(skip.keypoints(0, side))
            ka = set(zip(a["level"].tolist(), a["y"].tolist(), a["x"].tolist()))
            kb = set(zip(b["level"].tolist(), b["y"].tolist(), b["x"].tolist()))
            inter += len(ka & kb); total += len(ka); kept += len(kb)
    recall = inter / total
    print(f"{kind}: recall {recall:.4f} precision {inter / max(kept, 1):.4f} cells skipped {np.mean(skipped):.3f}")
    assert recall >= 0.99, (recall, inter / max(kept, 1))
    exact.close(); skip.close()
