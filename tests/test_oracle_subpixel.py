"""Pins of the oracle's correlation minimisation (Sec. III middle-end stereo
matching, read as patch-SAD refinement with a parabola fit): scenes whose
true disparity is known, integer and fractional, and the closed-form depth."""
import numpy as np
import pytest

from parity_util import params_from


def smooth_texture(H, W, shift, seed):
    """A band-limited texture T sampled at (x + shift, y): the right image of
    a fronto-parallel scene at disparity `shift` (a scene point at left
    column x is at right column x - shift), exact for any real shift."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    x = x + shift
    t = np.full((H, W), 128.0)
    for _ in range(7):
        fx, fy = rng.uniform(-0.45, 0.45, 2)
        amp = rng.uniform(12, 30)
        t += amp * np.sin(fx * x + fy * y + rng.uniform(0, 2 * np.pi))
    return np.clip(np.round(t), 0, 255).astype(np.uint8)


def blocky(H, W, seed):
    rng = np.random.default_rng(seed)
    b = rng.integers(30, 226, (H // 6 + 2, W // 6 + 2))
    img = np.kron(b, np.ones((6, 6)))[:H, :W]
    img += rng.integers(-12, 13, (H, W))
    return np.clip(img, 0, 255).astype(np.uint8)


def _run(oracle, left, right, levels=1, bf=0.0, **kw):
    p = params_from(oracle, levels=levels, max_feats=1500, fast_thresh=15, max_disp=64, match_max_dist=80, **kw)
    kl, kr, m = oracle.extract_pair(left, right, p)
    r = oracle.subpixel(left, right, kl, kr, m[0], p, 5, 5, bf)
    return kl, m, r


def test_integer_shift_is_found_exactly(oracle):
    """Noise-free right image = left shifted by 12 columns: at level 0 the
    SAD vanishes at the true alignment, so every surviving match has SAD 0
    and a disparity within half a pixel of 12."""
    H, W, d = 240, 360, 12
    base = blocky(H, W + d, 3)
    left, right = base[:, :W].copy(), base[:, d:d + W].copy()
    kl, m, r = _run(oracle, left, right)
    ok = r["disparity"] >= 0
    assert ok.sum() > 30
    assert (r["sad"][ok] == 0).all()
    assert np.abs(r["disparity"][ok] - d).max() < 0.5


def test_fractional_shift_is_refined(oracle):
    """A smooth scene at disparity 10.25: the refined disparity is closer to
    10.25 than the integer descriptor match can be (>= 0.25 away)."""
    H, W, d = 240, 360, 10.25
    left = smooth_texture(H, W, 0.0, 5)
    right = smooth_texture(H, W, d, 5)
    kl, m, r = _run(oracle, left, right)
    ok = r["disparity"] >= 0
    assert ok.sum() > 50
    err = np.abs(r["disparity"][ok] - d)
    assert np.median(err) < 0.15
    assert np.mean(err < 0.25) > 0.8


def test_depth_closed_form_and_rejections(oracle):
    H, W, d = 240, 360, 12
    base = blocky(H, W + d, 4)
    left, right = base[:, :W].copy(), base[:, d:d + W].copy()
    bf = np.float32(386.1448)
    kl, m, r = _run(oracle, left, right, levels=3, bf=float(bf))
    ok = r["disparity"] >= 0
    assert ok.any()
    np.testing.assert_allclose(r["depth"][ok] * np.maximum(r["disparity"][ok], 0.01), bf, rtol=1e-6)
    assert (r["depth"][~ok] == 0).all()
    # keypoints without a descriptor match get no SAD at all
    assert (r["sad"][m[0] < 0] == 0xFFFFFFFF).all()
    assert (r["disparity"][m[0] < 0] == -1).all()


def test_levels_scale_the_disparity(oracle):
    """At deeper levels the same scene disparity is found in s0 pixels (a
    band-limited scene, so that the resampled levels stay faithful)."""
    H, W, d = 300, 420, 16
    left = smooth_texture(H, W, 0.0, 6)
    right = smooth_texture(H, W, float(d), 6)
    kl, m, r = _run(oracle, left, right, levels=4)
    lev = kl["level"][: kl["count"]]
    ok = r["disparity"] >= 0
    for n in range(1, 4):
        sel = ok & (lev == n)
        if sel.sum() < 5:
            continue
        s = 1.2 ** n
        assert np.median(np.abs(r["disparity"][sel] - d)) < 0.5 * s, n


def test_brightness_offset_is_cancelled(oracle):
    """Each patch is taken relative to its centre pixel, so a right image
    brighter by a constant still correlates perfectly at the true shift
    (every earlier stage is offset-invariant: ring differences, BRIEF
    comparisons, resampling and blur weights summing to a power of two)."""
    H, W, d = 240, 360, 12
    base = blocky(H, W + d, 7)
    assert base.max() + 15 <= 255
    left, right = base[:, :W].copy(), (base[:, d:d + W] + 15).astype(np.uint8)
    kl, m, r = _run(oracle, left, right)
    ok = r["disparity"] >= 0
    assert ok.sum() > 30
    assert (r["sad"][ok] == 0).all()
