"""The seeded synthetic inputs have the properties the input recipe states:
the workload shapes, the checker scene's constant disparity, the planes
scene's disparity layout and its right image showing each left pixel at
x - d, the EuRoC-shaped scene's low-texture area, horizontal blur and gain
jumps, and determinism by seed."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes


def test_workload_table():
    w = scenes.WORKLOADS
    assert [(v["width"], v["height"], v["levels"], v["max_feats"]) for v in w.values()] == [
        (640, 480, 1, 300), (1241, 376, 8, 2000), (752, 480, 8, 1200), (1920, 1080, 8, 3000)]
    assert all(v["fast_thresh"] == 20 for v in w.values())
    assert [v["fast_thresh_lo"] for v in w.values()] == [0, 7, 7, 7]
    sizes = [(s["width"], s["height"], s["levels"]) for s in scenes.MIXED_STREAMS]
    assert sizes == [(640, 480, 4)] * 4 + [(752, 480, 5)] * 4 + [(1241, 376, 6)] * 4 + [(1920, 1080, 8)] * 4


def test_seeded_and_frames_differ():
    a, b = scenes.workload_pair("kitti_1241x376_L8", 3), scenes.workload_pair("kitti_1241x376_L8", 3)
    assert np.array_equal(a.left, b.left) and np.array_equal(a.right, b.right)
    c = scenes.workload_pair("kitti_1241x376_L8", 4)
    assert not np.array_equal(a.left, c.left)
    for p in (a, c):
        assert p.left.dtype == np.uint8 and p.left.shape == (376, 1241) and p.right.shape == (376, 1241)


def test_checker_has_constant_disparity_16():
    p = scenes.workload_pair("single_640x480_L1", 0)
    assert (p.disparity == 16).all()
    # right x shows left x + 16: equal up to the two images' independent noise (sigma 2 each)
    diff = p.right[:, :640 - 16].astype(int) - p.left[:, 16:].astype(int)
    assert np.median(np.abs(diff)) <= 2 and np.mean(np.abs(diff) <= 11) > 0.999
    # and not at another shift
    other = np.abs(p.right[:, :600].astype(int) - p.left[:, 24:624].astype(int))
    assert np.median(other) > 20


def test_planes_disparity_layout_and_right_image():
    p = scenes.workload_pair("kitti_1241x376_L8", 0)
    d = p.disparity
    H, W = d.shape
    assert d.min() == 0 and d.max() <= 96 and d.max() >= 80
    horizon = int(0.35 * H)
    # the background above the horizon is at disparity 0 outside the boxes: most of it
    assert np.mean(d[:horizon] == 0) > 0.5
    # the ground's disparity (the row's most common value) grows with the row below the horizon
    ground = [np.bincount(d[y]).argmax() for y in range(horizon + 1, H, 20)]
    assert all(b >= a for a, b in zip(ground, ground[1:])) and ground[-1] > ground[0]
    # a right pixel shows the left pixel's scene point at x - d (noise and occlusions aside)
    ys, xs = np.mgrid[0:H, 0:W]
    ok = xs - d >= 0
    diff = np.abs(p.right[ys[ok], (xs - d)[ok]].astype(int) - p.left[ok].astype(int))
    assert np.median(diff) <= 3 and np.mean(diff <= 11) > 0.9


def test_euroc_low_texture_blur_and_gain():
    frames = [scenes.workload_pair("euroc_752x480_L8", f) for f in (0, 25, 50, 75, 100, 125, 150, 175)]
    p = frames[0]
    assert p.left.shape == (480, 752) and p.disparity.max() <= 64
    img = p.left.astype(float)
    # low-texture regions: 8x8 blocks whose standard deviation is at most that of the noise and the
    # blurred sigma-3 texture cover about 30 % of the image or more
    blocks = img[:480 // 8 * 8, :752 // 8 * 8].reshape(60, 8, 94, 8).std(axis=(1, 3))
    assert np.mean(blocks <= 4.0) >= 0.25
    # horizontal box blur: horizontal differences are weaker than vertical ones
    assert np.abs(np.diff(img, axis=1)).mean() < 0.8 * np.abs(np.diff(img, axis=0)).mean()
    # gain jumps of +-20 % every 25 frames: the mean brightness takes at least two levels whose
    # ratio is near 1.2 or 1.5 (0.8, 1.0 and 1.2 in any pair)
    means = np.array([f.left.mean() for f in frames])
    r = means.max() / means.min()
    assert r > 1.12, means


def test_unknown_kind_is_refused():
    with pytest.raises(ValueError):
        scenes.stereo_pair("rings", 64, 64)
