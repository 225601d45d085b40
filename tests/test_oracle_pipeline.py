"""Pins of the oracle's whole-image pipeline (cap and canonical order) and of
its stereo matcher (Sec. III middle-end) by brute force and known-disparity
scenes."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes


def _params(oracle, **kw):
    p = oracle.FrontendParams()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_canonical_order_and_borders(oracle):
    img = scenes.random_image(200, 260, seed=4)
    p = _params(oracle, levels=4, max_feats=10000)
    kp = oracle.extract_image(img, p)
    n = kp["count"]
    assert n > 50
    key = kp["level"].astype(np.int64) << 32 | kp["y"].astype(np.int64) << 16 | kp["x"].astype(np.int64)
    assert np.all(np.diff(key) > 0)
    W, H, _ = oracle.level_geometry(260, 200, 4, 1.2, 32)
    for i in range(n):
        l = kp["level"][i]
        assert 19 <= kp["x"][i] < W[l] - 19 and 19 <= kp["y"][i] < H[l] - 19
        assert kp["X"][i] == oracle.project(int(kp["x"][i]), int(l), 1.2, 260)
        assert kp["Y"][i] == oracle.project(int(kp["y"][i]), int(l), 1.2, 200)


def test_cap_keeps_highest_priority(oracle):
    img = scenes.random_image(240, 320, seed=9)
    full = oracle.extract_image(img, _params(oracle, levels=5, max_feats=100000))
    n = full["count"]
    for cap in (1, 17, n // 2, n - 1):
        capped = oracle.extract_image(img, _params(oracle, levels=5, max_feats=cap))
        order = sorted(range(n), key=lambda i: (-int(full["k_levels"][i]), -int(full["k_resp"][i]),
                                               -int(full["response"][i]), int(full["level"][i]),
                                               int(full["y"][i]), int(full["x"][i])))
        want = sorted(order[:cap])  # canonical order == index order of `full`
        assert capped["count"] == cap
        for f in ("x", "y", "level", "response", "k_levels", "k_resp", "angle_bin"):
            assert np.array_equal(capped[f], full[f][want]), f
        assert np.array_equal(capped["desc"], full["desc"][want])


def test_lexicographic_rule_suppresses_a_superset(oracle):
    """Sec. II-C-2 NMS: a neighbour with larger K_l and larger K_r (rule 0)
    also has a lexicographically larger (K_l, K_r) (rule 1), and the scores
    do not depend on the rule, so without a cap rule 1 keeps a subset of
    rule 0's keypoints -- a proper one on a textured image."""
    img = scenes.random_image(240, 320, seed=9)
    key = lambda kp: set(zip(kp["level"].tolist(), kp["y"].tolist(), kp["x"].tolist()))
    a = key(oracle.extract_image(img, _params(oracle, levels=5, max_feats=100000)))
    b = key(oracle.extract_image(img, _params(oracle, levels=5, max_feats=100000, pfa_rule=1)))
    assert b < a


def _cap_cuts_hold(oracle, img, levels, pick):
    """Cut the cap inside ties of (K_l, K_r, response) chosen by `pick`: the
    capped set must be the first `cap` of the full set's priority order
    (K_l, K_r, response descending, then level, y, x ascending)."""
    full = oracle.extract_image(img, _params(oracle, levels=levels, max_feats=100000))
    n = full["count"]
    key = lambda i: (-int(full["k_levels"][i]), -int(full["k_resp"][i]), -int(full["response"][i]))
    order = sorted(range(n), key=lambda i: key(i) + (int(full["level"][i]), int(full["y"][i]), int(full["x"][i])))
    cuts = [c for c in range(1, n) if key(order[c - 1]) == key(order[c]) and pick(full, order[c - 1], order[c])]
    assert len(cuts) >= 3
    for cap in cuts[:6]:
        capped = oracle.extract_image(img, _params(oracle, levels=levels, max_feats=cap))
        want = sorted(order[:cap])
        for f in ("x", "y", "level"):
            assert np.array_equal(capped[f], full[f][want]), (cap, f)


def test_cap_breaks_ties_by_level_then_position(oracle):
    """Where (K_l, K_r, response) tie, a cap cutting inside the tie keeps the
    shallower level first, then the smaller y, then the smaller x.  Ties
    across levels come from a random image; ties within a level whose rows
    and columns are in opposite orders come from a texture tiled with the
    culling period (every cell repeats its strongest corner)."""
    _cap_cuts_hold(oracle, scenes.random_image(240, 320, seed=9), 5,
                   lambda f, a, b: f["level"][a] != f["level"][b])
    tiled = np.tile(scenes.random_image(32, 32, seed=9), (8, 10))
    _cap_cuts_hold(oracle, tiled, 3, lambda f, a, b: f["level"][a] == f["level"][b] and f["x"][a] > f["x"][b])


def test_cap_orders_by_summed_response_before_own_response(oracle):
    """Among keypoints with equal K_l, the cap keeps the larger K_r (summed over
    the levels) even when its own response is the smaller: a cap cut between
    such neighbours in the priority order."""
    img = scenes.random_image(240, 320, seed=9)
    p = _params(oracle, levels=5, max_feats=100000)
    full = oracle.extract_image(img, p)
    n = full["count"]
    pr = lambda i: (-int(full["k_levels"][i]), -int(full["k_resp"][i]), -int(full["response"][i]),
                    int(full["level"][i]), int(full["y"][i]), int(full["x"][i]))
    order = sorted(range(n), key=pr)
    cuts = [c for c in range(1, n) if full["k_levels"][order[c - 1]] == full["k_levels"][order[c]]
            and full["response"][order[c - 1]] < full["response"][order[c]]]
    assert len(cuts) >= 3
    for cap in cuts[:6]:
        capped = oracle.extract_image(img, _params(oracle, levels=5, max_feats=cap))
        want = sorted(order[:cap])
        for f in ("x", "y", "level"):
            assert np.array_equal(capped[f], full[f][want]), (cap, f)


def test_fallback_threshold_fills_cells_without_a_primary_corner(oracle):
    """One level (PFA never suppresses there): per 32x32 cell, the strongest
    corner at eps = 20 (response, then y, then x), or, in a cell without one,
    the strongest corner at eps_lo = 7 -- built here by brute force from the
    CRF-matrices at both thresholds (Eq. 1-3, pinned on their own)."""
    img = scenes.workload_pair("euroc_752x480_L8", 0).left
    H, W = img.shape
    kp = oracle.extract_image(img, _params(oracle, levels=1, max_feats=100000, fast_thresh_lo=7))
    hi, resp = oracle.fast(img, 20, 9, 13, 19)
    lo, _ = oracle.fast(img, 7, 9, 13, 19)
    want, from_lo = [], 0
    for cy in range(0, H, 32):
        for cx in range(0, W, 32):
            for flags, is_lo in ((hi, 0), (lo, 1)):
                ys, xs = np.nonzero(flags[cy:cy + 32, cx:cx + 32])
                if len(ys):
                    y, x = min(((cy + a, cx + b) for a, b in zip(ys, xs)), key=lambda t: (-int(resp[t]), t[0], t[1]))
                    want.append((y, x, int(resp[y, x])))
                    from_lo += is_lo
                    break
    got = sorted(zip(kp["y"].astype(int), kp["x"].astype(int), kp["response"].astype(int)))
    assert got == sorted(want)
    assert from_lo > 20  # the scene's flat regions leave cells to the fallback threshold
    # eps_lo = 0 turns the fallback off: only the primary-threshold selections
    kp0 = oracle.extract_image(img, _params(oracle, levels=1, max_feats=100000, fast_thresh_lo=0))
    got0 = sorted(zip(kp0["y"].astype(int), kp0["x"].astype(int), kp0["response"].astype(int)))
    assert len(got0) == len(want) - from_lo and set(got0) <= set(want)
    # eps_lo = 1 is a fallback threshold like any other
    kp1 = oracle.extract_image(img, _params(oracle, levels=1, max_feats=100000, fast_thresh_lo=1))
    got1 = set(zip(kp1["y"].astype(int), kp1["x"].astype(int)))
    assert set((y, x) for y, x, _ in got0) < got1


def test_orientation_uses_the_raw_level(oracle):
    """Level-0 keypoints: the intensity-centroid moments over the radius-15
    disk of the input image itself (the raw level, not the blurred one), by
    brute force here, and theta = atan2(m01, m10)."""
    img = scenes.random_image(200, 260, seed=4)
    kp = oracle.extract_image(img, _params(oracle, levels=3, max_feats=10000))
    dy, dx = np.mgrid[-15:16, -15:16]
    disk = dx * dx + dy * dy <= 225
    lv0 = np.nonzero(kp["level"] == 0)[0]
    assert len(lv0) > 20
    for i in lv0:
        x, y = int(kp["x"][i]), int(kp["y"][i])
        patch = img[y - 15:y + 16, x - 15:x + 16].astype(np.int64) * disk
        m10, m01 = int((dx * patch).sum()), int((dy * patch).sum())
        assert (kp["m10"][i], kp["m01"][i]) == (m10, m01)
        assert abs(float(kp["angle"][i]) - np.arctan2(m01, m10)) < 1e-6


def test_level0_sector_and_descriptor_by_brute_force(oracle):
    """Level-0 keypoints: the sector is the 12-degree sector of theta (away
    from exact boundaries), and the descriptor is BRIEF on the blurred input
    image with that sector's rotated pattern -- bit i = [B(p_i) < B(q_i)],
    bit i in word i / 32 -- computed here pair by pair."""
    img = scenes.random_image(200, 260, seed=4)
    kp = oracle.extract_image(img, _params(oracle, levels=3, max_feats=10000))
    blur = oracle.blur(img).astype(int)
    rot = oracle.pattern_rotated()
    lv0 = np.nonzero(kp["level"] == 0)[0]
    sectors = set()
    for i in lv0:
        x, y = int(kp["x"][i]), int(kp["y"][i])
        theta = np.arctan2(int(kp["m01"][i]), int(kp["m10"][i])) % (2 * np.pi)
        b = int(kp["angle_bin"][i])
        edge = theta / (2 * np.pi / 30)
        if abs(edge - round(edge)) > 1e-9:
            assert b == int(edge) % 30, (i, b, edge)
        sectors.add(b)
        want = np.zeros(8, np.uint32)
        for j, (px, py, qx, qy) in enumerate(rot[b].astype(int).tolist()):
            if blur[y + py, x + px] < blur[y + qy, x + qx]:
                want[j // 32] |= np.uint32(1 << (j % 32))
        assert np.array_equal(kp["desc"][i], want), i
    assert len(sectors) > 10


def test_pfa_reduces_keypoints_across_levels(oracle):
    """Sec. IV (PFA evaluation): aggregation lowers the feature count."""
    pair = scenes.workload_pair("kitti_1241x376_L8", 0)
    on = oracle.extract_image(pair.left, _params(oracle, max_feats=100000))
    off = oracle.extract_image(pair.left, _params(oracle, max_feats=100000, nms_q=1))
    assert on["count"] < off["count"]


def _brute_match(kl, kr, p, oracle):
    out = []
    for i in range(kl["count"]):
        band = oracle.match_band(int(kl["level"][i]), p.scale, p.row_band_px)
        best = None
        for j in range(kr["count"]):
            if abs(int(kr["level"][j]) - int(kl["level"][i])) > 1:
                continue
            if abs(int(kr["Y"][j]) - int(kl["Y"][i])) > band:
                continue
            d = int(kl["X"][i]) - int(kr["X"][j])
            if not 0 <= d <= p.max_disp:
                continue
            h = sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(kl["desc"][i], kr["desc"][j]))
            cand = (h, d, j)
            best = cand if best is None or cand < best else best
        if best is None:
            out.append((-1, 0, 0xFFFF))
        elif best[0] <= p.match_max_dist:
            out.append((best[2], best[1], best[0]))
        else:
            out.append((-1, 0, best[0]))
    return out


def test_match_brute_force(oracle):
    pair = scenes.planes_pair(400, 220, 0, 17, 18)
    for feats in (300, 100000):  # equal counts (capped), then different counts
        p = _params(oracle, levels=3, max_feats=feats, match_max_dist=90)
        kl, kr, (idx, disp, dist) = oracle.extract_pair(pair.left, pair.right, p)
        want = _brute_match(kl, kr, p, oracle)
        assert list(zip(idx.tolist(), disp.tolist(), dist.tolist())) == want
    assert kl["count"] != kr["count"]
    assert (idx >= 0).sum() > 20


def test_match_band_values(oracle):
    # ceil(2 * zeta^n) for zeta = 1.2: 2, 3, 3, 4, 5, 5, 6, 8
    assert [oracle.match_band(n, 1.2, 2) for n in range(8)] == [2, 3, 3, 4, 5, 5, 6, 8]


def test_known_disparity_scene(oracle):
    """Noise-free scene shifted by one cell (32 px): each cell of the left
    image sees the content of a right cell, the same corners are selected,
    and the matcher recovers the disparity."""
    pair = scenes.checker_pair(640, 480, seed=11, disparity=32, sigma=0.0)
    p = _params(oracle, levels=1, max_feats=300)
    kl, kr, (idx, disp, dist) = oracle.extract_pair(pair.left, pair.right, p)
    ok = idx >= 0
    assert ok.sum() > 200
    assert (disp[ok] == 32).mean() >= 0.97
    # epipolar: every accepted match lies in the row band and search range
    for i in np.nonzero(ok)[0]:
        j = idx[i]
        assert abs(int(kl["Y"][i]) - int(kr["Y"][j])) <= 2
        assert 0 <= int(kl["X"][i]) - int(kr["X"][j]) <= 128


def test_noisy_scene_low_distance_matches_are_right(oracle):
    pair = scenes.workload_pair("single_640x480_L1", 0)
    p = _params(oracle, levels=1, max_feats=300, match_max_dist=40)
    kl, kr, (idx, disp, dist) = oracle.extract_pair(pair.left, pair.right, p)
    ok = idx >= 0
    assert ok.sum() > 80
    assert (disp[ok] == 16).mean() >= 0.85


@pytest.mark.parametrize("bad", [dict(levels=0), dict(levels=9), dict(scale=1.0), dict(p_min=10, p_max=9),
                                 dict(cell=0), dict(nms_q=2), dict(border=10), dict(max_feats=0)])
def test_parameter_checks(oracle, bad):
    p = _params(oracle, **bad)
    assert not oracle.check_params(640, 480, p)
    assert oracle.check_params(640, 480, _params(oracle, levels=8))
    assert not oracle.check_params(60, 60, _params(oracle, levels=8))  # levels too small


def test_parameter_limits(oracle):
    """Each documented limit is accepted at its bound and rejected one past it;
    every level must keep 2 border + 1 pixels on each side."""
    def ok(W0=200, H0=200, **kw):
        return oracle.check_params(W0, H0, _params(oracle, **{"levels": 3, "max_feats": 100, **kw}))
    assert ok()
    for good, bad in [(dict(fast_thresh=1), dict(fast_thresh=0)), (dict(fast_thresh=254), dict(fast_thresh=255)),
                      (dict(fast_thresh_lo=254), dict(fast_thresh_lo=255)),
                      (dict(p_min=1, p_max=16), dict(p_max=17)), (dict(p_min=13, p_max=13), dict(p_min=14, p_max=13)),
                      (dict(cell=1), dict(cell=0)), (dict(cell=128), dict(cell=129)),
                      (dict(k_per_cell=8), dict(k_per_cell=9)), (dict(nms_q=7), dict(nms_q=9)),
                      (dict(nms_q=1), dict(nms_q=2)), (dict(border=16), dict(border=15)),
                      (dict(W0=4096), dict(W0=4097)), (dict(H0=4096), dict(H0=4097)),
                      (dict(levels=1), dict(levels=0)), (dict(levels=5), dict(levels=9)),
                      (dict(max_feats=1), dict(max_feats=0)), (dict(pfa_rule=1), dict(pfa_rule=2)),
                      (dict(pfa_rule=0), dict(pfa_rule=-1)), (dict(p_min=1), dict(p_min=0)),
                      (dict(k_per_cell=1), dict(k_per_cell=0)), (dict(nms_q=5), dict(nms_q=4)),
                      (dict(scale=1.01), dict(scale=1.0)),
                      # three levels: W_2 = round(W0 / 1.44) must be >= 39
                      (dict(W0=56), dict(W0=55)), (dict(H0=56), dict(H0=55))]:
        assert ok(**good), good
        assert not ok(**bad), bad
        # the whole-image extraction refuses the same parameters
        W0, H0 = bad.get("W0", 200), bad.get("H0", 200)
        if W0 <= 4096 and H0 <= 4096:
            kw = {k: v for k, v in bad.items() if k not in ("W0", "H0")}
            with pytest.raises(ValueError):
                oracle.extract_image(np.zeros((H0, W0), np.uint8), _params(oracle, **{"levels": 3, "max_feats": 100, **kw}))


def _hand_kps(X, Y, L, D):
    n = len(X)
    return {"count": n, "x": np.array(X, np.uint16), "y": np.array(Y, np.uint16), "X": np.array(X, np.uint16),
            "Y": np.array(Y, np.uint16), "level": np.array(L, np.uint8), "response": np.zeros(n, np.uint16),
            "k_levels": np.ones(n, np.uint8), "k_resp": np.zeros(n, np.uint32), "angle": np.zeros(n, np.float32),
            "angle_bin": np.zeros(n, np.uint8), "desc": np.array(D, np.uint32).reshape(n, 8)}


def test_match_hand_built(oracle):
    """Right keypoint 0 can be the match; a right keypoint to the right of the
    left one (negative disparity) is no candidate."""
    p = _params(oracle)
    z, five = [0] * 8, [0x1F] + [0] * 7
    kl = _hand_kps([100], [50], [0], [z])
    idx, disp, dist = oracle.match(kl, _hand_kps([90, 95], [50, 50], [0, 0], [z, five]), p)
    assert (idx[0], disp[0], dist[0]) == (0, 10, 0)
    idx, disp, dist = oracle.match(kl, _hand_kps([120], [50], [0], [z]), p)
    assert (idx[0], disp[0], dist[0]) == (-1, 0, 0xFFFF)
    # more right keypoints than left ones, the best at index 2; levels come
    # from each list (left levels 0 and 2; right keypoint 1 is at level 2)
    kl2 = _hand_kps([100, 100], [50, 50], [0, 2], [z, z])
    kr2 = _hand_kps([97, 92, 90], [50, 50, 50], [2, 0, 0], [z, z, five])
    idx, disp, dist = oracle.match(kl2, kr2, p)
    assert (idx[0], disp[0], dist[0]) == (1, 8, 0)    # right 0 (level 2) is outside left 0's band
    assert (idx[1], disp[1], dist[1]) == (0, 3, 0)    # level 2: right 0 only
    idx, disp, dist = oracle.match(kl, _hand_kps([95, 90], [50, 50], [0, 0], [five, z]), p)
    assert (idx[0], disp[0], dist[0]) == (1, 10, 0)   # the best right index is past the left list's length


def test_pipeline_composes_its_pinned_parts(oracle):
    """The whole-image extraction (no cap) equals its parts composed here:
    each level resampled (pinned on its own), its CRF at both thresholds,
    the cell culling, the s0 projection, then PFA by brute force -- K_l and
    K_r summed per s0 pixel, a keypoint suppressed by a q x q neighbour with
    larger K_l and larger K_r -- on a ragged, non-square image."""
    img = scenes.random_image(210, 333, seed=12)
    H0, W0 = img.shape
    p = _params(oracle, levels=4, max_feats=100000, fast_thresh_lo=7)
    kp = oracle.extract_image(img, p)
    W, H, c = oracle.level_geometry(W0, H0, p.levels, p.scale, p.cell)
    cand = []
    for n in range(p.levels):
        lvl = img if n == 0 else oracle.pyramid_level(img, p.scale, n)
        assert lvl.shape == (H[n], W[n])
        hi, resp = oracle.fast(lvl, p.fast_thresh, p.p_min, p.p_max, p.border)
        lo, _ = oracle.fast(lvl, p.fast_thresh_lo, p.p_min, p.p_max, p.border)
        xs, ys, rs = oracle.cull_level(hi, lo, resp, int(c[n]), p.k_per_cell)
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
        dominated = any(Kl.get((X + dx, Y + dy), 0) > kl and Kr.get((X + dx, Y + dy), 0) > kr
                        for dy in range(-rad, rad + 1) for dx in range(-rad, rad + 1) if dx or dy)
        if not dominated:
            want.append((n, y, x, X, Y, r, kl, kr))
    want.sort()
    got = list(zip(*(kp[f].astype(int).tolist() for f in ("level", "y", "x", "X", "Y", "response", "k_levels",
                                                          "k_resp"))))
    assert got == want
    assert len(set(lv for lv, *_ in want)) == p.levels and any(k > 1 for *_, k, _ in want)
