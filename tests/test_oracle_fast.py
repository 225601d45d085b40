"""Pins of the oracle's FAST + Bounded Rectification (Sec. II-A, Eq. 1-3)
against the paper's figures, brute force and closed forms."""
import itertools

import numpy as np
import pytest

from conftest import read_golden

pytestmark = pytest.mark.filterwarnings("ignore")

B = 19  # border used by the frontend


def test_ring_matches_paper_figure(oracle):
    rows = read_golden("ring_offsets.txt")
    dx, dy = oracle.ring()
    for idx, xs, ys in rows:
        k = int(idx)
        assert dx[k] == int(xs) and dy[k] == -int(ys), k
    # radius-3 Bresenham circle: 16 distinct points, neighbours 8-adjacent
    pts = set(zip(dx.tolist(), dy.tolist()))
    assert len(pts) == 16
    for k in range(16):
        j = (k + 1) % 16
        assert max(abs(dx[k] - dx[j]), abs(dy[k] - dy[j])) == 1
        assert 8 <= dx[k] ** 2 + dy[k] ** 2 <= 10


def _run_by_string(mask: int) -> int:
    if mask == 0xFFFF:
        return 16
    s = format(mask, "016b")
    return max(len(t) for t in (s + s).split("0"))


def test_longest_run_exhaustive(oracle):
    for m in range(1 << 16):
        assert oracle.longest_run(m) == _run_by_string(m), hex(m)


def test_corner_rule_from_masks(oracle):
    rng = np.random.default_rng(5)
    runs = {m: _run_by_string(m) for m in range(1 << 16)}
    ok = lambda m, lo, hi: lo <= runs[m] <= hi
    # every single mask against an empty partner, both roles
    for m in range(0, 1 << 16, 7):
        assert oracle.corner_from_masks(m, 0, 9, 13) == ok(m, 9, 13)
        assert oracle.corner_from_masks(0, m, 9, 13) == ok(m, 9, 13)
    # random disjoint (bright, dark) pairs; Eq. 3 read disjunctively
    for _ in range(20000):
        lab = rng.integers(0, 3, 16)
        bb = int(sum(1 << k for k in range(16) if lab[k] == 1))
        bd = int(sum(1 << k for k in range(16) if lab[k] == 2))
        want = ok(bb, 9, 13) or ok(bd, 9, 13)
        assert oracle.corner_from_masks(bb, bd, 9, 13) == want


def _ring_image(oracle, center: int, ring_vals, size: int = 2 * B + 1, fill=None):
    img = np.full((size, size), center if fill is None else fill, np.uint8)
    c = size // 2
    img[c, c] = center
    dx, dy = oracle.ring()
    for k in range(16):
        img[c + dy[k], c + dx[k]] = ring_vals[k]
    return img, c


def _label_center(oracle, img, c, eps=20, p_min=9, p_max=13):
    corner, resp = oracle.fast(img, eps, p_min, p_max, B)
    return bool(corner[c, c]), int(resp[c, c])


def test_noncorner_figure(oracle):
    rows = read_golden("noncorner_strip.txt")
    labels = [int(v) for v in rows[0]]
    classic_want, bounded_want = (int(v) for v in rows[1])
    ring_vals = [100 + 40 if l else 100 for l in labels]
    img, c = _ring_image(oracle, 100, ring_vals)
    classic, _ = _label_center(oracle, img, c, p_min=9, p_max=16)
    bounded, _ = _label_center(oracle, img, c, p_min=9, p_max=13)
    assert classic == bool(classic_want)
    assert bounded == bool(bounded_want)


@pytest.mark.parametrize("sign", [+1, -1])
@pytest.mark.parametrize("length,want", [(8, False), (9, True), (12, True), (13, True), (14, False), (16, False)])
def test_arcs(oracle, sign, length, want):
    for start in range(16):  # includes arcs that wrap 15 -> 0
        vals = [100] * 16
        for i in range(length):
            vals[(start + i) % 16] = 100 + sign * 40
        img, c = _ring_image(oracle, 100, vals)
        got, r = _label_center(oracle, img, c)
        assert got == want, (sign, length, start)
        assert r == 40 * length  # SAD over the whole circle


def test_threshold_equality_is_similar(oracle):
    # a 9-arc where one pixel differs by exactly eps is "similar" (Eq. 1 is strict)
    for sign in (+1, -1):
        vals = [100] * 16
        for i in range(9):
            vals[i] = 100 + sign * 30
        img, c = _ring_image(oracle, 100, vals)
        assert _label_center(oracle, img, c)[0]
        vals[4] = 100 + sign * 20
        img, c = _ring_image(oracle, 100, vals)
        assert not _label_center(oracle, img, c)[0]
        vals[4] = 100 + sign * 21
        img, c = _ring_image(oracle, 100, vals)
        assert _label_center(oracle, img, c)[0]


def test_single_bright_and_dark_pixel(oracle):
    # a lone bright pixel has an all-dark ring (N_d = 16): shot noise, rejected
    img, c = _ring_image(oracle, 200, [100] * 16, fill=100)
    assert _label_center(oracle, img, c) == (False, 1600)
    assert _label_center(oracle, img, c, p_max=16)[0]  # classic FAST accepts
    img, c = _ring_image(oracle, 10, [100] * 16, fill=100)
    assert _label_center(oracle, img, c) == (False, 1440)


def test_response_closed_form(oracle):
    rng = np.random.default_rng(3)
    for _ in range(50):
        center = int(rng.integers(40, 216))
        vals = rng.integers(0, 256, 16)
        img, c = _ring_image(oracle, center, vals.astype(np.uint8).tolist())
        _, r = _label_center(oracle, img, c)
        assert r == int(np.abs(vals.astype(int) - center).sum())


def test_border_is_skipped(oracle):
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (60, 70)).astype(np.uint8)
    corner, resp = oracle.fast(img, 20, 9, 13, B)
    assert corner[:B].sum() == 0 and corner[-B:].sum() == 0
    assert corner[:, :B].sum() == 0 and corner[:, -B:].sum() == 0
    assert resp[:B].sum() == 0 and resp[:, -B:].sum() == 0
    assert corner[B:-B, B:-B].sum() > 0


def test_brute_force_small_image(oracle):
    """Eq. 1-3 evaluated by plain Python on every pixel of a small image."""
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, (45, 47)).astype(np.uint8)
    img[10:30, 12:35] = rng.integers(90, 110, (20, 23))  # flatter region
    dx, dy = oracle.ring()
    for eps in (10, 20):
        corner, resp = oracle.fast(img, eps, 9, 13, B)
        for y, x in itertools.product(range(B, 45 - B), range(B, 47 - B)):
            ic = int(img[y, x])
            lab = ""
            for k in range(16):
                d = int(img[y + dy[k], x + dx[k]]) - ic
                lab += "b" if d > eps else ("d" if d < -eps else "s")
            best = 0
            for ch in "bd":
                s = "".join("1" if l == ch else "0" for l in lab)
                n = 16 if s == "1" * 16 else max(len(t) for t in (s + s).split("0"))
                best = best or (9 <= n <= 13)
            assert bool(corner[y, x]) == bool(best)
