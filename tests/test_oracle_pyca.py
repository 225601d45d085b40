"""Pins of the oracle's Feature Culling (Sec. II-C-1) and Pyramidal Feature
Aggregation (Sec. II-C-2, worked figure) by the paper's example, invariants
and brute force."""
import numpy as np
import pytest

from conftest import read_golden


def _cells(W, H, c):
    for cy in range((H + c - 1) // c):
        for cx in range((W + c - 1) // c):
            yield cx, cy, slice(cy * c, min(cy * c + c, H)), slice(cx * c, min(cx * c + c, W))


def _random_crf(rng, H, W, density):
    hi = (rng.random((H, W)) < density).astype(np.uint8)
    lo = np.maximum(hi, (rng.random((H, W)) < density * 2).astype(np.uint8))
    resp = rng.integers(1, 60, (H, W)).astype(np.uint16)  # small range: many ties
    return hi, lo, resp


@pytest.mark.parametrize("c,k", [(5, 1), (7, 2), (32, 1), (8, 3), (1, 1)])
def test_cull_against_brute_force(oracle, c, k):
    rng = np.random.default_rng(c * 10 + k)
    H, W = 45, 58  # ragged edge cells
    hi, lo, resp = _random_crf(rng, H, W, 0.05)
    for use_lo in (False, True):
        xs, ys, rs = oracle.cull_level(hi, lo if use_lo else None, resp, c, k)
        want = []
        for cx, cy, sy, sx in _cells(W, H, c):
            flags = hi[sy, sx]
            if flags.sum() == 0:
                if not use_lo:
                    continue
                flags = lo[sy, sx]
            yy, xx = np.nonzero(flags)
            yy = yy + sy.start; xx = xx + sx.start
            rr = resp[yy, xx].astype(int)
            order = sorted(range(len(rr)), key=lambda i: (-rr[i], yy[i], xx[i]))[:k]
            want += [(int(xx[i]), int(yy[i]), int(rr[i])) for i in order]
        assert list(zip(xs.tolist(), ys.tolist(), rs.tolist())) == want


def test_cull_invariants(oracle):
    rng = np.random.default_rng(21)
    H, W, c, k = 70, 90, 9, 2
    hi, lo, resp = _random_crf(rng, H, W, 0.1)
    xs, ys, rs = oracle.cull_level(hi, None, resp, c, k)
    cell = (ys // c) * ((W + c - 1) // c) + xs // c
    assert np.bincount(cell).max() <= k
    for x, y, r in zip(xs, ys, rs):
        assert hi[y, x] and resp[y, x] == r
        sy = slice((y // c) * c, (y // c) * c + c); sx = slice((x // c) * c, (x // c) * c + c)
        cand = resp[sy, sx][hi[sy, sx] > 0]
        # a survivor is among the k largest of its cell
        assert (cand > r).sum() < k
    # the selection does not depend on the visit order: with distinct
    # responses, culling the transposed CRF selects the transposed corners
    uniq = rng.permutation(H * W).reshape(H, W).astype(np.uint16) + 1
    xs1, ys1, _ = oracle.cull_level(hi, None, uniq, c, k)
    xs2, ys2, _ = oracle.cull_level(hi.T.copy(), None, uniq.T.copy(), c, k)
    assert sorted(zip(xs1.tolist(), ys1.tolist())) == sorted(zip(ys2.tolist(), xs2.tolist()))


def _load_pfa_example():
    rows = read_golden("pfa_example.txt")
    sec, kps, scores, surv = None, [], [], []
    for r in rows:
        if r[0] in ("keypoints", "scores", "survivors"):
            sec = r[0]
            continue
        v = [int(t) for t in r]
        {"keypoints": kps, "scores": scores, "survivors": surv}[sec].append(v)
    return kps, scores, surv


def test_pfa_paper_example(oracle):
    kps, scores, surv = _load_pfa_example()
    lev = [k[0] for k in kps]
    Y = [k[3] for k in kps]; X = [k[4] for k in kps]
    r = [k[5] for k in kps]
    Kl, Kr, alive = oracle.pfa_core(lev, X, Y, r, W0=5, H0=5, Ns=3, q=3, rule=0)
    want_scores = {(s[0], s[1]): (s[2], s[3]) for s in scores}
    for i in range(len(kps)):
        assert (Kl[i], Kr[i]) == want_scores[(Y[i], X[i])]
    kept = sorted((kps[i][0], kps[i][1], kps[i][2]) for i in range(len(kps)) if alive[i])
    assert kept == sorted(tuple(s) for s in surv)
    # the lexicographic alternative gives the same outcome on this example
    _, _, alive1 = oracle.pfa_core(lev, X, Y, r, W0=5, H0=5, Ns=3, q=3, rule=1)
    assert np.array_equal(alive, alive1)


def _pfa_brute(lev, X, Y, r, q, rule):
    score = {}
    for l, x, y, rr in zip(lev, X, Y, r):
        kl, kr = score.get((x, y), (0, 0))
        score[(x, y)] = (kl + 1, kr + rr)
    rad = (q - 1) // 2
    alive = []
    for x, y in zip(X, Y):
        kl, kr = score[(x, y)]
        dom = False
        for (qx, qy), (ql, qr) in score.items():
            if (qx, qy) == (x, y) or abs(qx - x) > rad or abs(qy - y) > rad:
                continue
            if rule == 0 and ql > kl and qr > kr:
                dom = True
            if rule == 1 and (ql, qr) > (kl, kr):
                dom = True
        alive.append(not dom)
    return score, alive


@pytest.mark.parametrize("rule", [0, 1])
@pytest.mark.parametrize("q", [1, 3, 5])
def test_pfa_brute_force(oracle, rule, q):
    rng = np.random.default_rng(100 + q + rule)
    W0, H0, Ns = 23, 17, 4
    lev, X, Y, r = [], [], [], []
    for n in range(Ns):
        pts = rng.choice(W0 * H0, 40, replace=False)  # one per pixel per level
        for p in pts:
            lev.append(n); X.append(int(p % W0)); Y.append(int(p // W0)); r.append(int(rng.integers(1, 50)))
    Kl, Kr, alive = oracle.pfa_core(lev, X, Y, r, W0, H0, Ns, q, rule)
    score, want = _pfa_brute(lev, X, Y, r, q, rule)
    assert alive.tolist() == want
    for i in range(len(lev)):
        assert (Kl[i], Kr[i]) == score[(X[i], Y[i])]
    if q == 1:
        assert alive.all()


def test_pfa_single_level_never_suppresses(oracle):
    rng = np.random.default_rng(8)
    pts = rng.choice(30 * 30, 200, replace=False)
    X = pts % 30; Y = pts // 30
    r = rng.integers(1, 100, len(pts))
    _, _, alive = oracle.pfa_core(np.zeros(len(pts), int), X, Y, r, 30, 30, 1, 3, 0)
    assert alive.all()


def test_projection_is_nearest(oracle):
    for n in range(8):
        s = oracle.level_scale(1.2, n)
        for x in range(0, 300, 7):
            X = oracle.project(x, n, 1.2, 10000)
            assert abs(X - x * s) <= 0.5 + 1e-9
    # distinct pixels of one level never share an s0 pixel
    for n in range(1, 8):
        Xs = [oracle.project(x, n, 1.2, 10000) for x in range(400)]
        assert len(set(Xs)) == 400


def test_equal_scores_do_not_suppress(oracle):
    """Sec. II-C-2 NMS suppresses only on a strictly larger score: under either
    rule, two neighbours with the same (K_l, K_r) both survive."""
    for rule in (0, 1):
        _, _, alive = oracle.pfa_core([0, 0], [10, 11], [10, 10], [50, 50], 30, 30, 1, q=3, rule=rule)
        assert alive.tolist() == [True, True], rule
    # and a larger K_r alone suppresses under rule 1 (equal K_l), not under rule 0
    for rule, want in ((0, [True, True]), (1, [False, True])):
        _, _, alive = oracle.pfa_core([0, 0], [10, 11], [10, 10], [50, 51], 30, 30, 1, q=3, rule=rule)
        assert alive.tolist() == want, rule
