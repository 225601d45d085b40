"""Host side of the Bounded Rectification repeatability study: the F1 score,
the labeled rotated scenes, and the study run on the oracle's corner sets
(Sec. IV-A, repeatability figure)."""
import numpy as np
import pytest

from paper_2410_04090_gb300 import repeatability as R
from paper_2410_04090_gb300 import scenes

W, H = R.SIZE


def test_f1_hand_cases():
    gt = np.array([[0.0, 0.0], [10.0, 0.0]])
    assert R.f1(gt.copy(), gt) == (1.0, 1.0, 1.0)
    assert R.f1(np.zeros((0, 2)), gt) == (0.0, 0.0, 0.0)
    assert R.f1(gt, np.zeros((0, 2))) == (0.0, 0.0, 0.0)
    # one detection near the first vertex, one far from both
    p, r, f = R.f1(np.array([[1.0, 1.0], [20.0, 0.0]]), gt)
    assert (p, r, f) == (0.5, 0.5, 0.5)
    # the radius is inclusive
    assert R.f1(np.array([[3.0, 0.0]]), gt[:1], radius=3.0)[2] == 1.0
    assert R.f1(np.array([[3.0 + 1e-9, 0.0]]), gt[:1], radius=3.0)[2] == 0.0
    # several detections around one vertex all count (sets, no assignment)
    p, r, f = R.f1(np.array([[0.5, 0.5], [-0.5, 0.5], [0.0, -1.0]]), gt)
    assert p == 1.0 and r == 0.5 and f == pytest.approx(2 / 3)


def test_f1_brute_force():
    rng = np.random.default_rng(4)
    for _ in range(20):
        det = rng.uniform(0, 40, (int(rng.integers(1, 30)), 2))
        gt = rng.uniform(0, 40, (int(rng.integers(1, 10)), 2))
        tp_d = sum(any(np.hypot(*(d - g)) <= 3.0 for g in gt) for d in det)
        tp_g = sum(any(np.hypot(*(g - d)) <= 3.0 for d in det) for g in gt)
        p, r = tp_d / len(det), tp_g / len(gt)
        want = 0.0 if p + r == 0 else 2 * p * r / (p + r)
        assert R.f1(det, gt) == pytest.approx((p, r, want))


def test_detections_are_pixel_centres():
    crf = np.zeros((5, 7), np.uint16)
    crf[1, 2] = 40
    crf[4, 6] = 7
    assert R.detections(crf).tolist() == [[2.5, 1.5], [6.5, 4.5]]


def test_scene_vertices_rotate_about_the_centre():
    base = scenes.corner_scene(W, H, 0, R.SEED).corners
    bg, shapes = scenes.corner_polygons(W, H, R.SEED)
    assert np.allclose(base, np.concatenate([v for v, _, _ in shapes]), atol=1e-9)
    cx, cy = W / 2, H / 2
    for a in (-175, -90, 25, 90, 150):
        got = scenes.corner_scene(W, H, a, R.SEED).corners
        t = np.radians(a)
        # counter-clockwise on screen with y down: (dx, dy) -> (dx cos + dy sin, -dx sin + dy cos)
        dx, dy = base[:, 0] - cx, base[:, 1] - cy
        want = np.stack([cx + dx * np.cos(t) + dy * np.sin(t), cy - dx * np.sin(t) + dy * np.cos(t)], axis=1)
        assert np.allclose(got, want, atol=1e-9)
    assert np.allclose(scenes.corner_scene(W, H, 30, R.SEED).corners,
                       scenes.corner_scene(W, H, 390, R.SEED).corners, atol=1e-9)


def test_scene_shapes_are_well_formed():
    bg, shapes = scenes.corner_polygons(W, H, R.SEED)
    assert len(shapes) == 14
    for i, (v, fill, (px, py, r)) in enumerate(shapes):
        assert abs(fill - bg) >= 40
        assert np.allclose(np.hypot(v[:, 0] - px, v[:, 1] - py), r)
        n = len(v)
        for k in range(n):  # interior angle at vertex k
            a, b, c = v[k - 1], v[k], v[(k + 1) % n]
            u, w = a - b, c - b
            ang = np.degrees(np.arccos(np.dot(u, w) / np.linalg.norm(u) / np.linalg.norm(w)))
            assert 30 - 1e-6 <= ang <= 150 + 1e-6
        for j in range(i):
            qx, qy, qr = shapes[j][2]
            assert np.hypot(px - qx, py - qy) >= r + qr + 6.0
    # every rotation keeps every vertex at least the margin from the edges
    for a in R.ANGLES:
        c = scenes.corner_scene(W, H, a, R.SEED).corners
        assert c[:, 0].min() >= 24 and c[:, 0].max() <= W - 24
        assert c[:, 1].min() >= 24 and c[:, 1].max() <= H - 24


def test_scene_pixels():
    s = scenes.corner_scene(W, H, 0, R.SEED)
    bg, shapes = scenes.corner_polygons(W, H, R.SEED)
    assert s.image.dtype == np.uint8 and s.image.shape == (H, W)
    assert abs(float(np.median(s.image[:10, :10])) - bg) <= 2  # the corners of the frame are background
    for v, fill, _ in shapes:  # the vertex centroid is inside the convex polygon
        mx, my = v.mean(axis=0)
        assert abs(int(s.image[int(my), int(mx)]) - fill) <= 10
    # the dots add pixels but no labeled corners
    d = scenes.corner_scene(W, H, 0, R.SEED, dots=40)
    assert np.array_equal(d.corners, s.corners)
    assert (d.image.astype(int) - s.image.astype(int) != 0).sum() > 40


@pytest.fixture(scope="module")
def oracle_sets(oracle):
    """Oracle corner sets of both detectors on both scene sets, five angles."""
    out = {}
    for set_name, dots in R.SCENES.items():
        for a in (-175, -50, 0, 75, 150):
            s = scenes.corner_scene(W, H, a, R.SEED, dots=dots)
            for name, p_max in R.P_MAX.items():
                c, resp = oracle.fast(s.image, 20, 9, p_max, 19)
                out[set_name, a, name] = (c.astype(bool), s.corners)
    return out


def test_bounded_corners_are_a_subset_of_plain_fast(oracle_sets):
    """Eq. 3 with P_max = 13 accepts a subset of the masks P_max = 16 accepts."""
    for (set_name, a, name), (c, _) in oracle_sets.items():
        if name == "bounded_rectification":
            plain = oracle_sets[set_name, a, "plain_fast"][0]
            assert not (c & ~plain).any()
            assert c.sum() > 0


def test_labeled_vertices_are_detectable(oracle_sets):
    """The scenes are fit for the study: with contrast >= 40 > eps = 20 and
    interior angles of 30-150 degrees, nearly every labeled vertex has a
    bounded-rectification corner within the radius."""
    for (set_name, a, name), (c, gt) in oracle_sets.items():
        ys, xs = np.nonzero(c)
        p, r, f = R.f1(np.stack([xs + 0.5, ys + 0.5], axis=1), gt)
        assert r >= 0.85, (set_name, a, name, r)
