"""The allocation-free entry point jslam_pfa_scores_static, for callers that
cannot allocate device memory (real-time loops that forbid allocation after
start-up, plug-ins inside another framework's enqueue hook, fixed memory
pools).

It gives the PFA scores (Sec. II-C-2) of a list of culled corners: for every
corner, its s0 projection, K_l, K_r and whether the NMS keeps it.  Checked
against the oracle's PFA for every corner of the list (suppressed ones
included) at q = 1, 3, 5, 7 under both rules; against the full extraction
(jslam_extract) for the corners it keeps; at the largest accepted list; with
inputs outside the domain (level >= levels, a response above 4080, a repeated
corner), which are marked and take no part; and for every argument it must
refuse.  Calls come several in a row, so the shared static scratch table is
cleared between calls.  This file is collected last."""
import ctypes as C

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


def _culled_corners(oracle, img, p):
    """Per-cell culled corners of every level of `img`: (level, x, y, response)."""
    H0, W0 = img.shape
    _, _, cells = oracle.level_geometry(W0, H0, p.levels, p.scale, p.cell)
    cols = [[], [], [], []]
    for n in range(p.levels):
        lvl = img if n == 0 else oracle.pyramid_level(img, p.scale, n)
        hi, resp = oracle.fast(lvl, p.fast_thresh, p.p_min, p.p_max, p.border)
        lo = oracle.fast(lvl, p.fast_thresh_lo, p.p_min, p.p_max, p.border)[0] if p.fast_thresh_lo > 0 else None
        xs, ys, rs = oracle.cull_level(hi, lo, resp, int(cells[n]), p.k_per_cell)
        cols[0] += [n] * len(xs); cols[1] += xs.tolist(); cols[2] += ys.tolist(); cols[3] += rs.tolist()
    return (np.array(cols[0], np.uint8), np.array(cols[1], np.uint16), np.array(cols[2], np.uint16),
            np.array(cols[3], np.uint16))


def _oracle_scores(oracle, lv, xs, ys, rs, W0, H0, levels, scale, q, rule):
    X = np.array([oracle.project(int(x), int(n), scale, W0) for x, n in zip(xs, lv)], np.int32)
    Y = np.array([oracle.project(int(y), int(n), scale, H0) for y, n in zip(ys, lv)], np.int32)
    Kl, Kr, alive = oracle.pfa_core(lv, X, Y, rs, W0, H0, levels, q, rule)
    return X, Y, Kl, Kr, alive


def _static(J, lv, xs, ys, rs, **kw):
    import torch
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (lv, xs, ys, rs)]
    out = J.pfa_scores_static(*t, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.fixture(scope="module")
def kitti_corners(oracle):
    pair = scenes.workload_pair("kitti_1241x376_L8", 5)
    p = params_from(oracle, levels=8, max_feats=8000, fast_thresh_lo=7)
    return pair, p, [_culled_corners(oracle, img, p) for img in (pair.left, pair.right)]


@pytest.mark.parametrize("q,rule", [(1, 0), (3, 0), (5, 0), (7, 0), (3, 1), (5, 1)])
def test_every_corner_scored_as_the_oracle_does(J, oracle, kitti_corners, q, rule):
    pair, p, corners = kitti_corners
    H0, W0 = pair.left.shape
    for lv, xs, ys, rs in corners:  # two calls in a row, on different lists
        X, Y, Kl, Kr, alive = _oracle_scores(oracle, lv, xs, ys, rs, W0, H0, p.levels, p.scale, q, rule)
        got = _static(J, lv, xs, ys, rs, width0=W0, height0=H0, levels=p.levels, scale=p.scale, nms_q=q,
                      pfa_rule=rule)
        assert np.array_equal(got["X"], X) and np.array_equal(got["Y"], Y)
        assert np.array_equal(got["k_levels"], Kl) and np.array_equal(got["k_resp"], Kr)
        assert np.array_equal(got["alive"], alive.astype(np.uint8))
        if q > 1:
            assert 0 < int((~alive).sum()) < len(alive)  # the NMS suppresses some, not all


@pytest.mark.parametrize("q,rule", [(3, 0), (5, 1)])
def test_kept_corners_match_extract(J, oracle, kitti_corners, q, rule):
    import torch
    pair, p0, corners = kitti_corners
    p = params_from(oracle, levels=8, max_feats=8000, fast_thresh_lo=7, nms_q=q, pfa_rule=rule)  # no cap
    fe = frontend_for(J, p, max_feats=8000)
    fe.extract(torch.from_numpy(pair.left).cuda(), torch.from_numpy(pair.right).cuda(),
               p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.sync()
    H0, W0 = pair.left.shape
    for side, (lv, xs, ys, rs) in enumerate(corners):
        kp = J.to_numpy(fe.keypoints(0, side))
        assert len(lv) > kp["count"] > 500
        out = _static(J, lv, xs, ys, rs, width0=W0, height0=H0, levels=p.levels, scale=p.scale, nms_q=q,
                      pfa_rule=rule)
        keep = out["alive"] == 1
        got = sorted(zip(lv[keep].tolist(), ys[keep].tolist(), xs[keep].tolist(), out["X"][keep].tolist(),
                         out["Y"][keep].tolist(), out["k_levels"][keep].tolist(), out["k_resp"][keep].tolist(),
                         rs[keep].tolist()))
        want = sorted(zip(kp["level"].tolist(), kp["y"].tolist(), kp["x"].tolist(), kp["X"].tolist(),
                          kp["Y"].tolist(), kp["k_levels"].tolist(), kp["k_resp"].tolist(),
                          kp["response"].tolist()))
        assert got == want, f"side {side}"
    fe.close()


def _random_corners(oracle, n, W0, H0, levels, scale, seed):
    """n distinct (level, x, y) inside their levels, with responses up to 4080."""
    rng = np.random.default_rng(seed)
    w, h, _ = oracle.level_geometry(W0, H0, levels, scale, 32)
    lv = rng.integers(0, levels, 4 * n)
    xs = (rng.random(4 * n) * w[lv]).astype(np.int64)
    ys = (rng.random(4 * n) * h[lv]).astype(np.int64)
    _, first = np.unique(np.stack([lv, ys, xs], 1), axis=0, return_index=True)
    pick = np.sort(rng.permutation(first)[:n])
    assert len(pick) == n
    rs = rng.integers(0, 4081, n)
    return lv[pick].astype(np.uint8), xs[pick].astype(np.uint16), ys[pick].astype(np.uint16), rs.astype(np.uint16)


def test_largest_list_accepted(J, oracle):
    W0, H0, levels, scale = 256, 192, 8, 1.2  # small, so that s0 pixels gather several levels
    lv, xs, ys, rs = _random_corners(oracle, 16384, W0, H0, levels, scale, 7)
    X, Y, Kl, Kr, alive = _oracle_scores(oracle, lv, xs, ys, rs, W0, H0, levels, scale, 3, 0)
    got = _static(J, lv, xs, ys, rs, width0=W0, height0=H0, levels=levels, scale=scale)
    assert Kl.max() >= 3  # dense enough that pixels gather several levels
    assert np.array_equal(got["X"], X) and np.array_equal(got["Y"], Y)
    assert np.array_equal(got["k_levels"], Kl) and np.array_equal(got["k_resp"], Kr)
    assert np.array_equal(got["alive"], alive.astype(np.uint8))


def test_inputs_outside_the_domain_are_marked(J, oracle):
    W0, H0, levels, scale = 256, 192, 4, 1.2
    lv, xs, ys, rs = _random_corners(oracle, 3000, W0, H0, levels, scale, 11)
    bad_level = np.array([4, 7, 255], np.uint8)
    lv2 = np.concatenate([lv, bad_level, lv[:2], lv[:5]])
    xs2 = np.concatenate([xs, xs[:3], xs[:2], xs[:5]])
    ys2 = np.concatenate([ys, ys[:3], ys[:2], ys[:5]])
    rs2 = np.concatenate([rs, rs[:3], np.array([4081, 65535], np.uint16), rs[:5]])
    # rows 3000..3002: level outside the pyramid; 3003..3004: responses above
    # 4080 (same corners as rows 0, 1: they must not count as repeats);
    # 3005..3009: repeats of rows 0..4
    got = _static(J, lv2, xs2, ys2, rs2, width0=W0, height0=H0, levels=levels, scale=scale, nms_q=5)
    X, Y, Kl, Kr, alive = _oracle_scores(oracle, lv, xs, ys, rs, W0, H0, levels, scale, 5, 0)
    a = got["alive"]
    assert (a[3000:3005] == 2).all()
    assert (got["X"][3000:3005] == 0xFFFF).all() and (got["k_resp"][3000:3005] == 0).all()
    # of each repeated pair one is marked 2 and the other scored as the oracle scores it
    for i in range(5):
        j = 3005 + i
        assert sorted([int(a[i]), int(a[j])])[1] == 2 and min(int(a[i]), int(a[j])) < 2
        s = i if a[i] < 2 else j
        assert (got["X"][s], got["Y"][s], got["k_levels"][s], got["k_resp"][s], a[s]) == \
            (X[i], Y[i], Kl[i], Kr[i], int(alive[i]))
    rest = np.arange(5, 3000)
    assert np.array_equal(got["k_levels"][rest], Kl[rest]) and np.array_equal(got["k_resp"][rest], Kr[rest])
    assert np.array_equal(a[rest], alive[rest].astype(np.uint8))


def test_refuses_bad_arguments(J):
    import torch
    z8 = torch.zeros(10, dtype=torch.uint8, device="cuda")
    z16 = torch.zeros(10, dtype=torch.uint16, device="cuda")
    ok = dict(width0=640, height0=480, levels=1)
    for bad, status in ((dict(levels=0), J.ERR_ARG), (dict(levels=9), J.ERR_ARG), (dict(scale=1.0), J.ERR_ARG),
                        (dict(scale=16.0), J.ERR_ARG), (dict(nms_q=2), J.ERR_ARG), (dict(nms_q=9), J.ERR_ARG),
                        (dict(pfa_rule=2), J.ERR_ARG), (dict(width0=4097), J.ERR_ARG), (dict(height0=0), J.ERR_ARG)):
        with pytest.raises(J.JslamError) as e:
            J.pfa_scores_static(z8, z16, z16, z16, **{**ok, **bad})
        assert e.value.status == status, bad
    big8 = torch.zeros(16385, dtype=torch.uint8, device="cuda")
    big16 = torch.zeros(16385, dtype=torch.uint16, device="cuda")
    with pytest.raises(J.JslamError) as e:
        J.pfa_scores_static(big8, big16, big16, big16, **ok)
    assert e.value.status == J.ERR_CAPACITY
    # through the C ABI directly: a negative count, a bad device, null arrays
    f = J.lib().jslam_pfa_scores_static
    p8, p16 = z8.data_ptr(), z16.data_ptr()
    args = lambda n, dev, ptr: (ptr, p16, p16, p16, n, 640, 480, 1, C.c_float(1.2), 3, 0, p16, p16, p8,
                                p16, p8, dev, None)
    assert f(*args(-1, 0, p8)) == J.ERR_ARG
    assert f(*args(10, -1, p8)) == J.ERR_ARG
    assert f(*args(10, 0, None)) == J.ERR_ARG
    assert f(*args(0, 0, None)) == J.OK  # nothing to do
    # the binding refuses mismatched inputs before any device work
    with pytest.raises(ValueError):
        J.pfa_scores_static(z8, z16[:9], z16, z16, **ok)
    with pytest.raises(ValueError):
        J.pfa_scores_static(z8, z16.to(torch.int32), z16, z16, **ok)
    with pytest.raises(ValueError):
        J.pfa_scores_static(z8, torch.zeros(20, dtype=torch.uint16, device="cuda")[::2], z16, z16, **ok)
