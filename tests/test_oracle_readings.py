"""Pins of the oracle's two off-by-default readings:

* the arc response (the alternative reading of Sec. III's "sum of absolute
  differences over the circle"): for each polarity whose longest circular
  run satisfies Eq. 3, the sum of (|d_k| - eps) over the ring positions on a
  run of that longest length; the larger sum of the two polarities;
* the cascaded pyramid (the alternative reading of the resampling): level n
  resampled from level n - 1 by one factor zeta instead of from level 0 by
  zeta^n.

Against closed forms, brute force written here in plain Python, and the
whole-image extraction composed from its separately pinned parts."""
import itertools

import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes

B = 19


def _labels(d, eps, sign):
    return [sign * dk > eps for dk in d]


def _longest(lab):
    if all(lab):
        return 16
    s = "".join("1" if v else "0" for v in lab)
    return max(len(t) for t in (s + s).split("0"))


def _arc_positions_ref(lab):
    n = _longest(lab)
    on = set()
    if n == 0:
        return on
    for start in range(16):
        if all(lab[(start + j) % 16] for j in range(n)):
            on.update((start + j) % 16 for j in range(n))
    return on


def _arc_response_ref(d, eps, p_min, p_max):
    best = 0
    for sign in (1, -1):
        lab = _labels(d, eps, sign)
        n = _longest(lab)
        if not (p_min <= n <= p_max) or n == 0:
            continue
        best = max(best, sum(abs(d[k]) - eps for k in _arc_positions_ref(lab)))
    return best


def _masks(d, eps):
    Bb = sum(1 << k for k in range(16) if d[k] > eps)
    Bd = sum(1 << k for k in range(16) if d[k] < -eps)
    return Bb, Bd


def test_arc_positions_exhaustive(oracle):
    """Positions on a run of maximal length, for every 16-bit mask."""
    for m in range(1 << 16):
        lab = [bool((m >> k) & 1) for k in range(16)]
        want = sum(1 << k for k in _arc_positions_ref(lab))
        assert oracle.arc_positions(m) == want, hex(m)


@pytest.mark.parametrize("d,eps,p_min,p_max,want", [
    # 9 bright pixels 30 above the centre at eps 20: 9 x 10
    ([30] * 9 + [0] * 7, 20, 9, 13, 90),
    # the same arc wrapping around position 0 (12..15, 0..4)
    ([30] * 5 + [0] * 7 + [30] * 4, 20, 9, 13, 90),
    # an arc of 12 dark pixels (-50) and a separate dark pixel: the arc only, 12 x 30
    ([-50] * 12 + [0, -50, 0, 0], 20, 9, 13, 360),
    # a run of 10 and a run of 3 of the same polarity: the run of 10 only
    ([25] * 10 + [0, 99, 99, 99, 0, 0], 20, 9, 13, 50),
    # the all-bright ring: no corner under Eq. 3 ...
    ([40] * 16, 20, 9, 13, 0),
    # ... but a corner of classic FAST (P_max = 16): all 16, 16 x 20
    ([40] * 16, 20, 9, 16, 320),
    # both polarities qualify at P_min = 8: the larger sum (8 x 30 > 8 x 10)
    ([50] * 8 + [-30] * 8, 20, 8, 13, 240),
    # a run of 14 is no corner for P_max 13
    ([30] * 14 + [0, 0], 20, 9, 13, 0),
    # |d| = eps is similar: the run is 8, not 9
    ([30] * 8 + [20] + [0] * 7, 20, 9, 13, 0),
])
def test_arc_response_closed_forms(oracle, d, eps, p_min, p_max, want):
    Bb, Bd = _masks(d, eps)
    assert oracle.arc_response(d, Bb, Bd, eps, p_min, p_max) == want
    assert _arc_response_ref(d, eps, p_min, p_max) == want


def test_arc_response_brute_force(oracle):
    rng = np.random.default_rng(3)
    for i in range(4000):
        # rings built from a few runs, so that corners are common
        d = np.zeros(16, np.int64)
        k = 0
        while k < 16:
            ln = int(rng.integers(1, 12))
            d[k:k + ln] = rng.integers(-120, 121)
            k += ln
        d = np.roll(d + rng.integers(-6, 7, 16), int(rng.integers(0, 16)))
        eps = int(rng.integers(1, 40))
        p_min = int(rng.integers(7, 12))
        p_max = int(rng.integers(p_min, 17))
        Bb, Bd = _masks(d.tolist(), eps)
        assert oracle.arc_response(d, Bb, Bd, eps, p_min, p_max) == \
            _arc_response_ref(d.tolist(), eps, p_min, p_max), (d.tolist(), eps, p_min, p_max)


def test_fast_arc_brute_force_small_image(oracle):
    """The arc CRF-matrix: the corners of fast(), the response of every corner
    by the definition above, 0 elsewhere and inside the border."""
    img = scenes.random_image(48, 50, seed=5)
    dx, dy = oracle.ring()
    b = 4
    for eps in (7, 20):
        corner0, _ = oracle.fast(img, eps, 9, 13, b)
        corner, resp = oracle.fast_arc(img, eps, 9, 13, b)
        assert np.array_equal(corner, corner0) and corner.sum() > 20
        for y, x in itertools.product(range(48), range(50)):
            if not (b <= y < 48 - b and b <= x < 50 - b):
                assert resp[y, x] == 0
                continue
            d = [int(img[y + dy[k], x + dx[k]]) - int(img[y, x]) for k in range(16)]
            want = _arc_response_ref(d, eps, 9, 13) if corner[y, x] else 0
            assert resp[y, x] == want, (y, x)


def _params(oracle, **kw):
    p = oracle.FrontendParams()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _compose(oracle, img, p, levels_of, crf_of):
    """Extraction without a cap composed from pinned parts: levels, CRF at
    both thresholds (crf_of returns corners and responses), cell culling,
    projection, brute-force PFA."""
    H0, W0 = img.shape
    W, H, c = oracle.level_geometry(W0, H0, p.levels, p.scale, p.cell)
    lv = levels_of(img, p)
    cand = []
    for n in range(p.levels):
        assert lv[n].shape == (H[n], W[n])
        hi, resp = crf_of(lv[n], p.fast_thresh, p)
        lo, resp_lo = crf_of(lv[n], p.fast_thresh_lo, p)
        merged = np.where(hi > 0, resp, resp_lo).astype(np.uint16)
        xs, ys, rs = oracle.cull_level(hi, lo, merged, int(c[n]), p.k_per_cell)
        for x, y, r in zip(xs.tolist(), ys.tolist(), rs.tolist()):
            cand.append((n, x, y, r, oracle.project(x, n, p.scale, W0), oracle.project(y, n, p.scale, H0)))
    Kl, Kr = {}, {}
    for n, x, y, r, X, Y in cand:
        Kl[X, Y] = Kl.get((X, Y), 0) + 1
        Kr[X, Y] = Kr.get((X, Y), 0) + r
    rad = (p.nms_q - 1) // 2
    want = []
    for n, x, y, r, X, Y in cand:
        kl, kr = Kl[X, Y], Kr[X, Y]
        if not any(Kl.get((X + ddx, Y + ddy), 0) > kl and Kr.get((X + ddx, Y + ddy), 0) > kr
                   for ddy in range(-rad, rad + 1) for ddx in range(-rad, rad + 1) if ddx or ddy):
            want.append((n, y, x, X, Y, r, kl, kr))
    return sorted(want)


def _got(kp):
    return list(zip(*(kp[f].astype(int).tolist() for f in ("level", "y", "x", "X", "Y", "response", "k_levels",
                                                            "k_resp"))))


def _direct_levels(oracle):
    return lambda img, p: [img if n == 0 else oracle.pyramid_level(img, p.scale, n) for n in range(p.levels)]


def _cascaded_levels(oracle):
    def levels(img, p):
        H0, W0 = img.shape
        W, H, _ = oracle.level_geometry(W0, H0, p.levels, p.scale, p.cell)
        out = [img]
        for n in range(1, p.levels):  # one factor zeta from the level above, at the level's own size
            out.append(oracle.pyramid_level_sized(out[-1], p.scale, 1, int(W[n]), int(H[n])))
        return out
    return levels


def test_arc_mode_extraction_composes(oracle):
    """response_mode = 1: primary-threshold corners ranked by their arc
    response at eps, the fallback corners of cells without one by theirs at
    the fallback threshold."""
    img = scenes.random_image(230, 320, seed=21)
    img[40:200, 60:250] = (img[40:200, 60:250] // 8 + 110).astype(np.uint8)  # low texture: fallback cells
    p = _params(oracle, levels=4, max_feats=100000, fast_thresh_lo=7, response_mode=1)
    kp = oracle.extract_image(img, p)
    arc = lambda lvl, eps, p: oracle.fast_arc(lvl, eps, p.p_min, p.p_max, p.border)
    want = _compose(oracle, img, p, _direct_levels(oracle), arc)
    assert _got(kp) == want
    # the fallback matters here: ranking fallback corners by the primary response changes the result
    wrong = _compose(oracle, img, p, _direct_levels(oracle),
                     lambda lvl, eps, p: (oracle.fast_arc(lvl, eps, p.p_min, p.p_max, p.border)[0],
                                          oracle.fast_arc(lvl, p.fast_thresh, p.p_min, p.p_max, p.border)[1]))
    assert wrong != want
    # and the arc reading is not the default reading
    assert _got(oracle.extract_image(img, _params(oracle, levels=4, max_feats=100000, fast_thresh_lo=7))) != want


def test_cascaded_levels(oracle):
    """Level 1 is the same either way; a constant image stays constant; at
    zeta = 2 a cascaded level is the rounded 2 x 2 mean of the level above."""
    img = scenes.random_image(200, 300, seed=4)
    W, H, _ = oracle.level_geometry(300, 200, 2, 1.2, 32)
    assert np.array_equal(oracle.pyramid_level_sized(img, 1.2, 1, int(W[1]), int(H[1])), oracle.pyramid_level(img, 1.2, 1))
    flat = np.full((120, 160), 77, np.uint8)
    lv = _cascaded_levels(oracle)(flat, _params(oracle, levels=5))
    assert all((l == 77).all() for l in lv)
    prev = scenes.random_image(64, 96, seed=9)
    half = oracle.pyramid_level_sized(prev, 2.0, 1, 48, 32)
    s = prev.astype(np.int64)
    mean = (s[0::2, 0::2] + s[0::2, 1::2] + s[1::2, 0::2] + s[1::2, 1::2] + 2) // 4
    assert np.array_equal(half, mean.astype(np.uint8))


def test_cascaded_mode_extraction_composes(oracle):
    """pyramid_mode = 1: the extraction on levels resampled one factor at a
    time, each from the level above; deeper levels differ from the direct
    reading, so the mode is not a no-op."""
    img = scenes.random_image(260, 350, seed=17)
    p = _params(oracle, levels=5, max_feats=100000, fast_thresh_lo=7, pyramid_mode=1)
    kp = oracle.extract_image(img, p)
    crf = lambda lvl, eps, p: oracle.fast(lvl, eps, p.p_min, p.p_max, p.border)
    want = _compose(oracle, img, p, _cascaded_levels(oracle), crf)
    assert _got(kp) == want
    cas = _cascaded_levels(oracle)(img, p)
    dirl = _direct_levels(oracle)(img, p)
    assert np.array_equal(cas[1], dirl[1]) and not np.array_equal(cas[3], dirl[3])
    assert want != _compose(oracle, img, p, _direct_levels(oracle), crf)


@pytest.mark.parametrize("field,value", [("response_mode", 2), ("response_mode", -1), ("pyramid_mode", 2)])
def test_mode_fields_are_checked(oracle, field, value):
    p = _params(oracle, **{field: value})
    assert not oracle.check_params(640, 480, p)
