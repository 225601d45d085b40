"""Pins of the oracle's correlation minimisation (Sec. III middle-end stereo
matching, read as patch-SAD refinement with a parabola fit): scenes whose
true disparity is known, integer and fractional, and the closed-form depth."""
import numpy as np

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


def _kps(x, y, level, X=None):
    n = len(x)
    X = x if X is None else X
    z8 = lambda: np.zeros(n, np.uint8)
    return {"count": n, "x": np.array(x, np.uint16), "y": np.array(y, np.uint16), "X": np.array(X, np.uint16),
            "Y": np.array(y, np.uint16), "level": np.array(level, np.uint8), "response": np.zeros(n, np.uint16),
            "k_levels": np.ones(n, np.uint8), "k_resp": np.zeros(n, np.uint32), "angle": np.zeros(n, np.float32),
            "angle_bin": z8(), "desc": np.zeros((n, 8), np.uint32)}


def _params(oracle, **kw):
    p = oracle.FrontendParams()
    p.levels, p.max_disp = 1, 64
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_first_minimum_of_tied_sads(oracle):
    """A texture periodic in x with period 4 and identical left and right
    images: SAD(t) vanishes at t = -4, 0 and 4 around xr0 = x.  The first
    minimum, t* = -4, gives the disparity 4 - delta (|delta| <= 1); the last
    one would give a negative disparity, which is rejected."""
    rng = np.random.default_rng(8)
    tile = rng.integers(20, 236, (40, 4))
    img = np.tile(tile, (1, 15)).astype(np.uint8)             # 40 x 60
    kl = _kps([30], [20], [0])
    r = oracle.subpixel(img, img, kl, _kps([30], [20], [0]), np.array([0]), _params(oracle), 5, 5)
    assert r["sad"][0] == 0
    assert 3.0 <= r["disparity"][0] <= 5.0


def _outlier_case(oracle, ks, d=3):
    """Right image = left shifted by d columns, then k pixels of the window of
    keypoint i (never its centre) raised by 1, so that SAD(t*) = k exactly."""
    rng = np.random.default_rng(9)
    H, W = 40, 25 * len(ks) + 25
    base = rng.integers(20, 230, (H, W + d))
    left, right = base[:, :W].copy(), base[:, d:d + W].copy()
    xs = [20 + 25 * i for i in range(len(ks))]
    # the window's corners and edge midpoints first, so that every SAD counts
    # its first and last rows and columns
    edges = [(5, 5), (5, -5), (-5, 5), (-5, -5), (5, 0), (0, 5), (-5, 0), (0, -5)]
    offsets = edges + [(dy, dx) for dy in range(-5, 6) for dx in range(-5, 6)
                       if (dy, dx) != (0, 0) and (dy, dx) not in edges]
    for x, k in zip(xs, ks):
        for dy, dx in offsets[:k]:
            right[20 + dy, x - d + dx] += 1
    left, right = left.astype(np.uint8), right.astype(np.uint8)
    n = len(ks)
    r = oracle.subpixel(left, right, _kps(xs, [20] * n, [0] * n), _kps([x - d for x in xs], [20] * n, [0] * n),
                        np.arange(n), _params(oracle), 5, 5)
    assert r["sad"].tolist() == list(ks)
    kept = r["disparity"] >= 0
    assert np.all(np.abs(r["disparity"][kept] - d) <= 1.0)
    return kept.tolist()


def test_outlier_bound_is_inclusive_at_21_tenths_of_the_median(oracle):
    """The median is element count / 2 of the kept SADs in ascending order; a
    match is an outlier when 10 SAD > 21 median.  Odd count: SADs 10, 10, 10,
    21, 22 have median 10, so 21 stays and 22 goes.  Even count: SADs 10, 10,
    20, 42 have median 20 (the upper one), so 42 stays (420 <= 420)."""
    assert _outlier_case(oracle, [10, 10, 10, 21, 22]) == [True, True, True, True, False]
    assert _outlier_case(oracle, [10, 10, 20, 42]) == [True, True, True, True]
    assert _outlier_case(oracle, [10, 10, 20, 43]) == [True, True, True, False]
    # the median is taken in SAD order, not in keypoint order
    assert _outlier_case(oracle, [22, 10, 21, 10, 10]) == [False, True, True, True, True]


def test_search_centre_is_the_nearest_level_column(oracle):
    """Scale 1.25 (exact Q8 weights): a right image shifted by 5 level-0
    columns is shifted by exactly 4 columns at level 1.  For the level-1 left
    keypoint x = 41 the true right column is 37; the match's s0 column
    X = 41 gives xr0 = round(41 / 1.25) = 33, so the minimum lies at t* = 4,
    inside the search of +-5 (rounding down, xr0 = 32, would put it at the
    edge t* = 5 and reject it)."""
    rng = np.random.default_rng(10)
    H0, W0 = 60, 120
    base = rng.integers(0, 256, (H0, W0 + 5))
    left, right = base[:, :W0].astype(np.uint8), base[:, 5:W0 + 5].astype(np.uint8)
    p = _params(oracle, levels=2, scale=1.25)
    l1, r1 = oracle.pyramid_level(left, 1.25, 1), oracle.pyramid_level(right, 1.25, 1)
    assert np.array_equal(r1[:, :80], l1[:, 4:84])          # the exact 4-column shift at level 1
    r = oracle.subpixel(left, right, _kps([41], [24], [1]), _kps([41], [24], [1]), np.array([0]), p, 5, 5)
    assert r["sad"][0] == 0
    assert abs(r["disparity"][0] - 1.25 * 4) <= 1.25


def test_windows_must_fit_inside_the_level(oracle):
    """The left (2w+1)^2 window and the right strip (columns xr0 +- (L + w))
    must lie inside the level: a keypoint whose window ends on the first or
    last column or row is evaluated, one pixel further it is rejected with no
    SAD (w = L = 5, a 60 x 40 level)."""
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, (40, 60)).astype(np.uint8)
    NONE = 0xFFFFFFFF

    def sad(x, y, X):
        r = oracle.subpixel(img, img, _kps([x], [y], [0]), _kps([X], [y], [0]), np.array([0]), _params(oracle), 5, 5)
        return int(r["sad"][0])
    assert sad(54, 20, 44) != NONE and sad(55, 20, 44) == NONE   # x + w = 59 fits, 60 does not
    assert sad(30, 34, 30) != NONE and sad(30, 35, 30) == NONE   # y + w = 39 fits, 40 does not
    assert sad(5, 20, 15) != NONE and sad(4, 20, 15) == NONE     # x - w = 0 fits, -1 does not
    assert sad(30, 5, 30) != NONE and sad(30, 4, 30) == NONE     # y - w = 0 fits, -1 does not
    assert sad(30, 20, 49) != NONE and sad(30, 20, 50) == NONE   # xr0 + L + w = 59 fits, 60 does not
    assert sad(30, 20, 10) != NONE and sad(30, 20, 9) == NONE    # xr0 - L - w = 0 fits, -1 does not


def test_minimum_at_either_end_of_the_search_is_rejected(oracle):
    """Right image = left shifted by 3 columns, so left column 30 is right
    column 27 and t* = 27 - xr0 (xr0 = X at level 0).  A minimum at t = -L or
    t = +L may lie beyond the search and is rejected (its SAD still reported);
    one step inside it is kept, at disparity 3 - delta."""
    rng = np.random.default_rng(12)
    base = rng.integers(0, 256, (40, 63))
    left, right = base[:, :60].astype(np.uint8), base[:, 3:63].astype(np.uint8)

    def run(X):
        r = oracle.subpixel(left, right, _kps([30], [20], [0]), _kps([X], [20], [0]), np.array([0]),
                            _params(oracle), 5, 5)
        return int(r["sad"][0]), float(r["disparity"][0])
    assert run(32) == (0, -1.0)                 # t* = -5 = -L
    assert run(22) == (0, -1.0)                 # t* = +5 = +L
    for X in (31, 23):                          # t* = -4 and +4
        sad, d = run(X)
        assert sad == 0 and 2.0 <= d <= 4.0


def test_disparity_bounds_are_inclusive(oracle):
    """A texture mirror-symmetric about the keypoint's column gives SAD(t* - 1)
    = SAD(t* + 1), so delta = 0 and the disparity is an exact integer: 0 for
    identical images, D for a right image shifted by D.  Both ends of
    [0, max_disp] are kept (max_disp = D = 6)."""
    rng = np.random.default_rng(13)
    H, W, D = 40, 61, 6
    B = rng.integers(0, 256, (H, W + D))
    B[:, :61] = np.concatenate([B[:, :30], B[:, 30:31], B[:, :30][:, ::-1]], axis=1)  # symmetric about 30
    left, right = B[:, :W].astype(np.uint8), B[:, D:D + W].astype(np.uint8)
    p = _params(oracle, max_disp=D)
    r = oracle.subpixel(left, left, _kps([30], [20], [0]), _kps([30], [20], [0]), np.array([0]), p, 5, 5)
    assert r["sad"][0] == 0 and r["disparity"][0] == 0.0
    r = oracle.subpixel(left, right, _kps([30], [20], [0]), _kps([30 - D], [20], [0]), np.array([0]), p, 5, 5)
    assert r["sad"][0] == 0 and r["disparity"][0] == float(D)


def test_negative_refined_disparity_is_rejected(oracle):
    """Identical images: the true disparity is 0 and the refined one is
    -delta, so a match is kept exactly when delta <= 0."""
    ks = [0] * 8
    free = _outlier_disparities(oracle, ks, max_disp=64, d=0)
    assert ((free == -1.0).sum() >= 2) and ((free >= 0).sum() >= 2)
    rng = np.random.default_rng(9)
    H, W = 40, 25 * len(ks) + 25
    img = rng.integers(20, 230, (H, W)).astype(np.int64)
    for i, x in enumerate(20 + 25 * k for k in range(len(ks))):
        lp = img[15:26, x - 5:x + 6] - img[20, x]
        sad = [int(np.abs(lp - (img[15:26, x + t - 5:x + t + 6] - img[20, x + t])).sum()) for t in (-1, 0, 1)]
        delta = (sad[0] - sad[2]) / (2 * (sad[0] + sad[2] - 2 * sad[1]))
        assert (free[i] >= 0) == (delta <= 0), (i, delta, free[i])


def test_max_disparity_is_tested_on_the_refined_value(oracle):
    """Right image = left shifted by 3 columns and max_disp = 3: a match is
    kept exactly when its refined disparity 3 - delta is at most 3, i.e. when
    delta >= 0 -- the bound applies to the sub-pixel value, not to the
    integer shift or to 3 + delta."""
    ks = [0] * 8
    free = _outlier_disparities(oracle, ks, max_disp=64)
    capped = _outlier_disparities(oracle, ks, max_disp=3)
    assert (free > 3.0).any() and (free < 3.0).any()          # both signs of delta occur
    assert np.array_equal(capped >= 0, free <= 3.0)
    assert np.array_equal(capped[capped >= 0], free[free <= 3.0])


def _outlier_disparities(oracle, ks, max_disp, d=3):
    rng = np.random.default_rng(9)
    H, W = 40, 25 * len(ks) + 25
    base = rng.integers(20, 230, (H, W + d))
    left, right = base[:, :W].astype(np.uint8), base[:, d:d + W].astype(np.uint8)
    xs = [20 + 25 * i for i in range(len(ks))]
    n = len(ks)
    r = oracle.subpixel(left, right, _kps(xs, [20] * n, [0] * n), _kps([x - d for x in xs], [20] * n, [0] * n),
                        np.arange(n), _params(oracle, max_disp=max_disp), 5, 5)
    return r["disparity"]


def test_refinement_against_brute_force(oracle):
    """The SAD curve over shifts -L..L of the centre-normalised windows, its
    first minimum, the parabola vertex delta = (d1 - d3) / (2 (d1 + d3 - 2 d2))
    and the disparity x - xr0 - t* - delta, all computed here from their
    definitions in numpy for keypoints of a random scene shifted by 3."""
    rng = np.random.default_rng(14)
    H, W, d, w, L = 40, 230, 3, 5, 5
    base = rng.integers(0, 256, (H, W + d))
    left, right = base[:, :W].astype(np.uint8), base[:, d:d + W].astype(np.uint8)
    right[15:26, :] = np.clip(right[15:26, :].astype(int) + rng.integers(-6, 7, (11, W)), 0, 255)
    xs = [20 + 25 * i for i in range(8)]
    Xr = [x - d + o for x, o in zip(xs, (0, 1, -1, 2, -2, 0, 1, -1))]
    r = oracle.subpixel(left, right, _kps(xs, [20] * 8, [0] * 8), _kps(Xr, [20] * 8, [0] * 8), np.arange(8),
                        _params(oracle), w, L)
    A, B = left.astype(np.int64), right.astype(np.int64)
    n_ok, kept_sads, want_disp = 0, [], {}
    for i, (x, xr0) in enumerate(zip(xs, Xr)):
        lp = A[20 - w:21 + w, x - w:x + w + 1] - A[20, x]
        sad = [int(np.abs(lp - (B[20 - w:21 + w, xr0 + t - w:xr0 + t + w + 1] - B[20, xr0 + t])).sum())
               for t in range(-L, L + 1)]
        k = int(np.argmin(sad))                      # first minimum
        assert r["sad"][i] == sad[k]
        if k in (0, 2 * L):
            assert r["disparity"][i] == -1.0
            continue
        d1, d2, d3 = sad[k - 1], sad[k], sad[k + 1]
        delta = (d1 - d3) / (2 * (d1 + d3 - 2 * d2))
        want_disp[i] = x - xr0 - (k - L) - delta
        kept_sads.append(sad[k])
    # outliers: 10 SAD > 21 median, the median being element count / 2 of the
    # kept SADs in ascending order
    median = sorted(kept_sads)[len(kept_sads) // 2]
    for i, want in want_disp.items():
        if 10 * int(r["sad"][i]) > 21 * median:
            assert r["disparity"][i] == -1.0
            continue
        assert abs(float(r["disparity"][i]) - want) <= 1e-6 * max(1.0, abs(want)), (i, r["disparity"][i], want)
        n_ok += 1
    assert n_ok >= 6


def test_matches_are_looked_up_through_right_idx(oracle):
    """Each left keypoint is refined against the right keypoint its match
    names, on the left keypoint's level: two left keypoints whose matches are
    listed in the other order, a right list longer than the left one whose
    entries carry other levels, and an unmatched left keypoint (-1)."""
    rng = np.random.default_rng(15)
    H, W, d = 40, 120, 3
    base = rng.integers(0, 256, (H, W + d))
    left, right = base[:, :W].astype(np.uint8), base[:, d:d + W].astype(np.uint8)
    kl = _kps([30, 70, 50], [20, 20, 20], [0, 0, 0])
    kr = _kps([67, 27, 5, 90], [20, 20, 20, 20], [1, 1, 1, 1])   # 70 - 3 and 30 - 3, then two others
    r = oracle.subpixel(left, right, kl, kr, np.array([1, 0, -1]), _params(oracle), 5, 5)
    assert r["sad"][0] == 0 and r["sad"][1] == 0 and r["sad"][2] == 0xFFFFFFFF
    assert np.all(np.abs(r["disparity"][:2] - d) <= 1.0) and r["disparity"][2] == -1.0


def test_outlier_rule_covers_every_left_keypoint(oracle):
    """Two left keypoints at the same place share one right keypoint (SAD 22
    each) after three with SAD 10: the rule runs over the left list, so both
    late ones are rejected although the right list is shorter."""
    rng = np.random.default_rng(9)
    H, W, d = 40, 125, 3
    base = rng.integers(20, 230, (H, W + d))
    left, right = base[:, :W].copy(), base[:, d:d + W].copy()
    xs = [20, 45, 70, 95]
    edges = [(5, 5), (5, -5), (-5, 5), (-5, -5), (5, 0), (0, 5), (-5, 0), (0, -5)]
    offsets = edges + [(dy, dx) for dy in range(-5, 6) for dx in range(-5, 6)
                       if (dy, dx) != (0, 0) and (dy, dx) not in edges]
    for x, k in zip(xs, (10, 10, 10, 22)):
        for dy, dx in offsets[:k]:
            right[20 + dy, x - d + dx] += 1
    left, right = left.astype(np.uint8), right.astype(np.uint8)
    kl = _kps(xs + [95], [20] * 5, [0] * 5)
    kr = _kps([x - d for x in xs], [20] * 4, [0] * 4)
    r = oracle.subpixel(left, right, kl, kr, np.array([0, 1, 2, 3, 3]), _params(oracle), 5, 5)
    assert r["sad"].tolist() == [10, 10, 10, 22, 22]
    assert (r["disparity"] >= 0).tolist() == [True, True, True, False, False]
