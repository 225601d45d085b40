"""The repeatability study on the GPU: the CRF-matrix read through
jslam_crf_view equals the oracle's corner response bit for bit (both
detectors, both scene sets, rotated scenes), and the study's F1 values are
the ones the oracle's corner sets give."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import repeatability as R
from paper_2410_04090_gb300 import scenes

pytestmark = pytest.mark.gpu

W, H = R.SIZE
ANGLES = (-175, -50, 0, 75, 150)


@pytest.fixture(scope="module")
def J():
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


@pytest.mark.parametrize("set_name", list(R.SCENES))
@pytest.mark.parametrize("detector", list(R.P_MAX))
def test_crf_matches_oracle(J, oracle, set_name, detector):
    import torch
    p_max, dots = R.P_MAX[detector], R.SCENES[set_name]
    sc = [scenes.corner_scene(W, H, a, R.SEED, dots=dots) for a in ANGLES]
    imgs = [torch.from_numpy(s.image).cuda() for s in sc]
    fe = J.Frontend(max_width=W, max_height=H, max_feats=4000, max_pairs=len(sc), p_min=9, p_max=p_max, border=19,
                    fast_thresh_lo=0)
    jobs = fe.prepare_batch([J.Job(im, im, levels=1, scale=1.2, fast_thresh=20, cell=32, max_feats=4000)
                             for im in imgs])
    fe.extract_batch(jobs)
    fe.fc_ablation(8)
    fe.sync()
    for i, s in enumerate(sc):
        got = fe.crf(i, 0, 0).cpu().numpy().astype(np.int64)
        c, resp = oracle.fast(s.image, 20, 9, p_max, 19)
        want = np.where(c > 0, resp, 0).astype(np.int64)
        assert got.shape == (H, W)
        assert np.array_equal(got, want), (set_name, detector, ANGLES[i], np.argwhere(got != want)[:3])
        # the right image is the same frame: its CRF is the same
        assert np.array_equal(fe.crf(i, 1, 0).cpu().numpy().astype(np.int64), want)
    fe.close()


def test_study_f1_equals_oracle(J, oracle):
    res = R.study(angles=ANGLES)
    for set_name, dots in R.SCENES.items():
        for name, p_max in R.P_MAX.items():
            for k, a in enumerate(ANGLES):
                s = scenes.corner_scene(W, H, a, R.SEED, dots=dots)
                c, _ = oracle.fast(s.image, 20, 9, p_max, 19)
                ys, xs = np.nonzero(c)
                want = R.f1(np.stack([xs + 0.5, ys + 0.5], axis=1), s.corners)
                got = (res[set_name][name]["precision"][k], res[set_name][name]["recall"][k],
                       res[set_name][name]["f1"][k])
                assert got == want, (set_name, name, a)
    assert res["crf_ms"] > 0


def test_crf_view_errors(J):
    import torch
    fe = J.Frontend(max_width=W, max_height=H, max_feats=100, max_pairs=1)
    with pytest.raises(RuntimeError):
        fe.crf(0, 0, 0)  # no ablation yet
    im = torch.from_numpy(scenes.corner_scene(W, H, 0, R.SEED).image).cuda()
    fe.extract(im, im, levels=2, scale=1.2, fast_thresh=20, cell=32, max_feats=100)
    fe.fc_ablation(8)
    fe.sync()
    for bad in ((1, 0, 0), (0, 2, 0), (0, 0, 2), (0, 0, -1)):
        with pytest.raises(RuntimeError):
            fe.crf(*bad)
    assert tuple(fe.crf(0, 0, 1).shape) == (round(H / 1.2), round(W / 1.2))
    fe.close()
