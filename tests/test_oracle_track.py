"""Pins of the oracle's feature tracking by projection (Sec. III middle-end:
feature tracking with projected map points): a frame tracks its own
keypoints, a known image translation is recovered, and the window, level
band, distance threshold and ratio test behave as their definitions fix."""
import numpy as np

from paper_2410_04090_gb300 import scenes
from parity_util import params_from


def _frame(oracle, img, **kw):
    p = params_from(oracle, levels=5, max_feats=1500, fast_thresh_lo=7, **kw)
    return oracle.extract_image(img, p), p


def _queries(kp):
    n = kp["count"]
    return (kp["X"][:n].astype(np.float32), kp["Y"][:n].astype(np.float32), kp["level"][:n].copy(),
            np.asarray(kp["desc"])[:n].copy())


def test_frame_tracks_itself(oracle):
    img = scenes.planes_pair(480, 360, 0, 11, 12).left
    kp, p = _frame(oracle, img)
    u, v, lv, d = _queries(kp)
    idx, dist = oracle.track(kp, p.scale, u, v, lv, d, radius=0.5)
    n = kp["count"]
    assert (dist == 0).all()                      # every query finds its own keypoint
    self_hit = idx == np.arange(n)
    assert self_hit.mean() > 0.95                 # rejected only by an ambiguous second candidate
    assert (idx[~self_hit] == -1).all()


def test_translation_is_recovered(oracle):
    """The next frame is the same image shifted by (+7, -4) pixels: queries
    predicted at the old positions plus the shift find keypoints at that
    offset (level 0, where a pixel shift is an exact keypoint shift).  The
    culling grid does not move with the content, so some cells keep other
    corners; every zero-distance match (identical descriptor, the same
    content) is exactly at the shift."""
    base = scenes.random_image(400, 520, 21)
    a = base[10:370, 20:500].copy()
    b = base[14:374, 13:493].copy()   # content moves by (+7, -4)
    ka, p = _frame(oracle, a)
    kb, _ = _frame(oracle, b)
    u, v, lv, d = _queries(ka)
    sel = lv == 0
    idx, dist = oracle.track(kb, p.scale, u[sel] + 7, v[sel] - 4, lv[sel], d[sel], radius=3.0)
    ok = idx >= 0
    assert ok.mean() > 0.6
    dx = kb["X"][idx[ok]].astype(int) - ka["X"][: ka["count"]][sel][ok].astype(int)
    dy = kb["Y"][idx[ok]].astype(int) - ka["Y"][: ka["count"]][sel][ok].astype(int)
    exact = (dx == 7) & (dy == -4)
    assert exact.mean() > 0.7
    zero = dist[ok] == 0
    assert zero.sum() > 50 and exact[zero].all()


def test_window_level_band_threshold_and_ratio(oracle):
    """Hand-built keypoint lists: the window is inclusive at r, levels outside
    n +- 1 are ignored, max_dist bounds the best distance, and two equally
    good candidates fail the 0.9 ratio test."""
    def kps(X, Y, L, D):
        n = len(X)
        return {"count": n, "x": np.array(X, np.uint16), "y": np.array(Y, np.uint16),
                "X": np.array(X, np.uint16), "Y": np.array(Y, np.uint16), "level": np.array(L, np.uint8),
                "response": np.zeros(n, np.uint16), "k_levels": np.ones(n, np.uint8),
                "k_resp": np.zeros(n, np.uint32), "angle": np.zeros(n, np.float32),
                "angle_bin": np.zeros(n, np.uint8), "desc": np.array(D, np.uint32).reshape(n, 8)}
    z = [0] * 8
    one = [1] + [0] * 7          # distance 1 from z
    far = [0xFFFFFFFF] * 4 + [0] * 4  # distance 128
    kf = kps([100, 110, 100, 300, 300], [50, 50, 60, 40, 40], [0, 0, 3, 0, 0], [one, z, z, z, z])
    q = lambda u, v, l, d, r, md=100: oracle.track(kf, 1.2, [u], [v], [l], [d], r, md)
    assert q(100, 50, 0, z, 10.0)[0][0] == 1       # k1 (distance 0) beats k0 (1); k2 is at level 3
    assert q(100, 50, 0, z, 9.5)[0][0] == 0        # k1 at |dx| = 10 > 9.5: only k0 (k2 level 3 is out of band)
    assert q(90, 50, 0, z, 10.0)[0][0] == 0        # |dx| = 10 = r for k0 is inside; k1 at 20 is not
    assert q(100, 50, 2, z, 10.0)[0][0] == 2       # level 2 +- 1 admits level 3 only (r = 10 * 1.44)
    assert tuple(x[0] for x in q(500, 50, 0, z, 10.0)) == (-1, 0xFFFF)  # no candidate
    i, d = q(300, 40, 0, z, 1.0)                    # k3 and k4 identical: ratio 0 / 0 passes (10*0 <= 9*0)
    assert i[0] == 3 and d[0] == 0
    i, d = q(300, 40, 0, one, 1.0)                  # both at distance 1: 10 > 9 rejects
    assert i[0] == -1 and d[0] == 1
    i, d = q(100, 50, 0, far, 10.0, 100)            # best distance 127 > max_dist
    assert i[0] == -1 and d[0] == 127


def test_ratio_bound_second_best_and_scaled_window(oracle):
    """The ratio test is inclusive at 0.9 (distances 18 and 20 pass, 19 and 21
    fail); a better candidate met later makes the earlier best the second;
    the window's half-size at level n is radius * zeta^n."""
    def bits(k):  # a descriptor at Hamming distance k from the zero descriptor
        d = np.zeros(8, np.uint32)
        for i in range(k):
            d[i // 32] |= np.uint32(1 << (i % 32))
        return d

    def kps(X, L, D):
        n = len(X)
        return {"count": n, "x": np.array(X, np.uint16), "y": np.full(n, 50, np.uint16),
                "X": np.array(X, np.uint16), "Y": np.full(n, 50, np.uint16), "level": np.array(L, np.uint8),
                "response": np.zeros(n, np.uint16), "k_levels": np.ones(n, np.uint8),
                "k_resp": np.zeros(n, np.uint32), "angle": np.zeros(n, np.float32),
                "angle_bin": np.zeros(n, np.uint8), "desc": np.stack(D).astype(np.uint32)}
    z = np.zeros(8, np.uint32)
    q = lambda kf, lvl, r: tuple(int(a[0]) for a in oracle.track(kf, 1.2, [100.0], [50.0], [lvl], [z], r, 100))
    assert q(kps([100, 101], [0, 0], [bits(18), bits(20)]), 0, 5.0) == (0, 18)   # 180 <= 180
    assert q(kps([100, 101], [0, 0], [bits(19), bits(21)]), 0, 5.0) == (-1, 19)  # 190 > 189
    assert q(kps([100, 101], [0, 0], [bits(20), bits(19)]), 0, 5.0) == (-1, 19)  # 20 became the second
    assert q(kps([100, 101, 102], [0, 0, 0], [bits(30), bits(19), bits(20)]), 0, 5.0) == (-1, 19)
    far = kps([112], [2], [bits(3)])  # |dx| = 12 at level 2
    assert q(far, 2, 10.0) == (0, 3)                # r = 10 * 1.44 = 14.4 >= 12
    assert q(far, 2, 8.0) == (-1, 0xFFFF)           # r = 8 * 1.44 = 11.52 < 12
    assert q(far, 1, 10.0) == (0, 3)                # level 1 +- 1 admits level 2; r = 12.0, inclusive
    assert q(far, 0, 100.0) == (-1, 0xFFFF)         # level 0 +- 1 does not admit level 2
    deep = kps([100], [7], [bits(2)])
    assert q(deep, 7, 1.0) == (0, 2)
    # the band rule at any level: 8 +- 1 admits level 7 with r = zeta^8 = 4.30, 9 +- 1 admits none
    assert q(deep, 8, 1.0) == (0, 2)
    assert q(deep, 9, 1.0) == (-1, 0xFFFF)
    deep4 = kps([104], [7], [bits(2)])              # |dx| = 4 at level 7
    assert q(deep4, 8, 1.0) == (0, 2)               # r = 4.30 >= 4
    assert q(deep4, 8, 0.9) == (-1, 0xFFFF)         # r = 3.87 < 4
    assert q(kps([100], [3], [bits(2)]), 4, 1.0) == (0, 2)   # level 4 - 1 is in the band
    one = kps([100], [0], [bits(3)])
    t = lambda v, md: tuple(int(a[0]) for a in oracle.track(one, 1.2, [100.0], [v], [0], [z], 5.0, md))
    assert t(45.0, 100) == (0, 3) and t(44.5, 100) == (-1, 0xFFFF)   # |dy| = 5 = r is inside
    assert t(50.0, 3) == (0, 3) and t(50.0, 2) == (-1, 3)            # max_dist is inclusive
    last = np.zeros(8, np.uint32)
    last[7] = np.uint32(0xF0000000)                                   # 4 bits in the last word
    assert q(kps([100], [0], [last]), 0, 5.0) == (0, 4)
