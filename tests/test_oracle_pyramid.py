"""Pins of the oracle's level geometry, pyramid resampling and Gaussian blur
(Sec. III, streamlined multiscale detection and extraction)."""
import numpy as np
import pytest
from scipy import ndimage

from conftest import read_golden


def test_cell_scaling_matches_paper(oracle):
    for c0, scale, level, want in read_golden("cell_scaling.txt"):
        W, H, c = oracle.level_geometry(1241, 376, int(level) + 1, float(scale), int(c0))
        assert c[int(level)] == int(want)
        assert c[0] == int(c0)


def test_cells_never_shrink_below_one_pixel(oracle):
    """c_n = max(1, floor(c / zeta^n)): for c = 2 the floor is 0 from
    level 4 (2 / 1.2^4 = 0.96) on, and the cell stays one pixel."""
    _, _, c = oracle.level_geometry(1241, 376, 8, 1.2, 2)
    assert c.tolist() == [2, 1, 1, 1, 1, 1, 1, 1]
    _, _, c = oracle.level_geometry(1241, 376, 8, 1.2, 1)
    assert c.tolist() == [1] * 8


def test_level_sizes_shrink_by_scale(oracle):
    for W0, H0 in ((1241, 376), (752, 480), (1920, 1080), (640, 480)):
        W, H, _ = oracle.level_geometry(W0, H0, 8, 1.2, 32)
        assert W[0] == W0 and H[0] == H0
        s = np.array([oracle.level_scale(1.2, n) for n in range(8)])
        # nearest integer to W0 / zeta^n
        assert np.all(np.abs(W - W0 / s) <= 0.5 + 1e-9)
        assert np.all(np.abs(H - H0 / s) <= 0.5 + 1e-9)
        assert np.all(np.diff(W) < 0) and np.all(np.diff(H) < 0)


def test_constant_image_stays_constant(oracle):
    img = np.full((120, 150), 77, np.uint8)
    for n in range(1, 8):
        lvl = oracle.pyramid_level(img, 1.2, n)
        assert np.all(lvl == 77)
    assert np.all(oracle.blur(img) == 77)


def _reference_bilinear(img, n, Wn, Hn, scale=1.2):
    """Bilinear resampling by scipy at pixel-centre-aligned positions."""
    H0, W0 = img.shape
    s = float(np.float64(np.float32(scale)) ** n)
    u = np.clip((np.arange(Wn) + 0.5) * s - 0.5, 0, W0 - 1)
    v = np.clip((np.arange(Hn) + 0.5) * s - 0.5, 0, H0 - 1)
    vv, uu = np.meshgrid(v, u, indexing="ij")
    return ndimage.map_coordinates(img.astype(np.float64), [vv, uu], order=1, mode="nearest")


def test_bilinear_against_scipy(oracle):
    rng = np.random.default_rng(11)
    img = ndimage.gaussian_filter(rng.integers(0, 256, (97, 131)).astype(np.float64), 1.0)
    img = np.clip(img, 0, 255).astype(np.uint8)
    for n in range(1, 8):
        lvl = oracle.pyramid_level(img, 1.2, n)
        ref = _reference_bilinear(img, n, lvl.shape[1], lvl.shape[0])
        # Q8 weights move the value by at most 255/512 per axis, plus rounding
        assert np.max(np.abs(lvl - ref)) <= 1.5


def _q8_bound(img, n, Wn, Hn, scale=1.2):
    """Per output pixel: 1/2 (rounding to nearest) + (dx + dy) / 512, where dx
    and dy are the largest horizontal and vertical differences of the 2x2
    source cell holding the exact position: Q8 weights are each within 1/512
    of the exact fractions, and the bilinear interpolant changes by at most
    dx (dy) per unit of its horizontal (vertical) argument in that cell."""
    H0, W0 = img.shape
    s = float(np.float64(np.float32(scale)) ** n)
    u = np.clip((np.arange(Wn) + 0.5) * s - 0.5, 0, W0 - 1)
    v = np.clip((np.arange(Hn) + 0.5) * s - 0.5, 0, H0 - 1)
    xa = np.floor(u).astype(int); xb = np.minimum(xa + 1, W0 - 1)
    ya = np.floor(v).astype(int); yb = np.minimum(ya + 1, H0 - 1)
    I = img.astype(np.int64)
    p00, p01 = I[np.ix_(ya, xa)], I[np.ix_(ya, xb)]
    p10, p11 = I[np.ix_(yb, xa)], I[np.ix_(yb, xb)]
    dx = np.maximum(np.abs(p01 - p00), np.abs(p11 - p10))
    dy = np.maximum(np.abs(p10 - p00), np.abs(p11 - p01))
    return 0.5 + (dx + dy) / 512.0 + 1e-9


def test_bilinear_within_the_q8_error_bound(oracle):
    """The level equals the exact bilinear value (scipy) to within the bound
    that Q8 weights rounded to nearest and a final rounding to nearest allow.
    A smooth image makes the bound close to 1/2 (rounding down instead would
    break it); vertical step edges of 0 and 255 make it close to 1 (weights
    truncated instead of rounded would break it)."""
    y, x = np.mgrid[0:157, 0:211]
    smooth = np.round(128 + 60 * np.sin(x / 9.0) * np.cos(y / 11.0)).astype(np.uint8)
    rng = np.random.default_rng(5)
    cols = np.cumsum(rng.integers(1, 6, 211)) % 2  # 0/255 columns in random runs
    steps = np.repeat((cols * 255).astype(np.uint8)[None, :], 157, axis=0)
    for scale in (1.2, 1.1, 1.37, 1.63):
        for img in (smooth, steps):
            for n in range(1, 8 if scale < 1.5 else 4):
                lvl = oracle.pyramid_level(img, scale, n)
                ref = _reference_bilinear(img, n, lvl.shape[1], lvl.shape[0], scale)
                bound = _q8_bound(img, n, lvl.shape[1], lvl.shape[0], scale)
                assert np.all(np.abs(lvl - ref) <= bound), (scale, n, float(np.max(np.abs(lvl - ref) - bound)))


def test_scale_two_is_the_rounded_2x2_mean(oracle):
    """At zeta = 2 every level-1 pixel centre lies exactly between four level-0
    centres (u = 2x + 1/2, weights 128/256), so bilinear resampling is the 2x2
    box mean rounded half up, (sum + 2) div 4 -- with many exact ties."""
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (64, 90)).astype(np.uint8)
    lvl = oracle.pyramid_level(img, 2.0, 1)
    H, W = lvl.shape
    assert (H, W) == (32, 45)
    I = img.astype(int)
    s = I[0:2 * H:2, 0:2 * W:2] + I[1:2 * H:2, 0:2 * W:2] + I[0:2 * H:2, 1:2 * W:2] + I[1:2 * H:2, 1:2 * W:2]
    assert np.array_equal(lvl, (s + 2) // 4)
    assert ((s % 4) == 2).sum() > 100


def test_blur_rounds_half_up_at_exact_ties(oracle):
    """Two pixels on a zero image put the blurred centre exactly on a half
    (82 at the centre and 244 beside it: (54*54*82 + 54*49*244) / 65536 = 13.5,
    so 14) and just below one (138 at the centre and 119 diagonal:
    (54*54*138 + 49*49*119) / 65536 = 10.49998..., so 10)."""
    for pix, want in (({(7, 7): 82, (7, 8): 244}, 14), ({(7, 7): 138, (8, 8): 119}, 10)):
        img = np.zeros((15, 15), np.uint8)
        for (y, x), v in pix.items():
            img[y, x] = v
        out = oracle.blur(img)
        assert out[7, 7] == want
        w = oracle.blur_weights() / 256.0
        ref = ndimage.convolve1d(ndimage.convolve1d(img.astype(np.float64), w, axis=1, mode="nearest"), w, axis=0,
                                 mode="nearest")
        assert np.array_equal(out, np.floor(ref + 0.5).astype(np.uint8))


def test_pyramid_preserves_mirror_symmetry(oracle):
    """Pixel-centre alignment maps the image centre onto the level centre:
    a left-right mirror-symmetric image stays mirror symmetric (to rounding)."""
    rng = np.random.default_rng(2)
    half = rng.integers(0, 256, (24, 864)).astype(np.uint8)
    img = np.concatenate([half, half[:, ::-1]], axis=1)  # 1728 = 1000 * 1.2^3
    tested = 0
    for n in range(1, 8):
        lvl = oracle.pyramid_level(img, 1.2, n).astype(int)
        # exact only where the level is an exact scaled copy (W_n zeta^n = W0)
        if abs(lvl.shape[1] * oracle.level_scale(1.2, n) - 1728) < 1e-3:
            assert np.max(np.abs(lvl - lvl[:, ::-1])) <= 1
            tested += 1
    assert tested == 3
    # a mapping without the half-pixel alignment (u = x zeta^n) breaks it
    s = oracle.level_scale(1.2, 1)
    u = np.arange(1440) * s
    shifted = np.interp(u, np.arange(1728), img[0].astype(float))
    assert np.max(np.abs(shifted - shifted[::-1])) > 10


def test_blur_weights_and_scipy(oracle):
    w = oracle.blur_weights()
    assert w.tolist() == [18, 34, 49, 54, 49, 34, 18]
    g = np.exp(-np.arange(-3, 4) ** 2 / 8.0)
    # each outer tap is rounded to the nearest 1/256; the centre tap also
    # absorbs the residual so the weights sum to exactly 256
    assert np.max(np.abs(w / 256.0 - g / g.sum())[[0, 1, 2, 4, 5, 6]]) <= 0.5 / 256
    assert abs(w[3] / 256.0 - 1 / g.sum()) < 1.5 / 256 and w.sum() == 256
    rng = np.random.default_rng(4)
    img = rng.integers(0, 256, (40, 53)).astype(np.uint8)
    out = oracle.blur(img)
    ref = ndimage.convolve1d(img.astype(np.float64), w / 256.0, axis=1, mode="nearest")
    ref = ndimage.convolve1d(ref, w / 256.0, axis=0, mode="nearest")
    assert np.array_equal(out, np.floor(ref + 0.5).astype(np.uint8))


def test_blur_is_symmetric(oracle):
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, (33, 41)).astype(np.uint8)
    a = oracle.blur(img)
    b = oracle.blur(img[:, ::-1].copy())[:, ::-1]
    c = oracle.blur(img[::-1].copy())[::-1]
    assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.parametrize("W0,H0", [(64, 48), (1241, 376)])
def test_level_zero_of_pyramid_is_input(oracle, W0, H0):
    # the first panel of the pipeline: level 0 raw is the input; the oracle's
    # resampler at zeta^0 = 1 reproduces it exactly (u = x, weights 0)
    rng = np.random.default_rng(W0)
    img = rng.integers(0, 256, (H0, W0)).astype(np.uint8)
    assert np.array_equal(oracle.pyramid_level(img, 1.2, 0), img)
