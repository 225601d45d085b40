"""Seeded synthetic stereo scenes shaped like the paper's workloads.

This module only makes inputs: it holds none of the frontend's arithmetic.
Both the CUDA path's tests/benchmark and the CPU oracle consume what it
produces.  Every array comes from ``numpy.random.Generator(PCG64(seed))``.

Workloads (the paper's datasets are not available, so these stand in for
their shapes and statistics):

* ``kind="checker"``  640x480-style: an 8 px checkerboard (64/192) overlaid
  with random polygons (3-8 vertices, uniform fill), constant disparity
  (16 px by default), Gaussian noise sigma = 2 (the single-pair workload).
* ``kind="planes"``   KITTI-shaped (1241x376) and larger: a ground plane whose
  disparity grows linearly with the row (0..96 px below the horizon), a far
  background at disparity 0 and fronto-parallel textured boxes, the camera
  translating 0.5 px per frame, noise sigma = 2.
* ``kind="euroc"``    EuRoC-shaped (752x480): the planes scene with 30 % of the
  area replaced by low-texture regions (texture sigma <= 3), a horizontal box
  motion blur of 5-15 px per frame and global gain jumps of +/-20 % every 25
  frames.

A right image pixel x shows the scene point that the left image shows at
x + d, so disparity d = x_left - x_right >= 0.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache

import numpy as np

# The five workload shapes (width, height, kind, levels, max_feats, eps, eps_lo).
WORKLOADS = {
    "single_640x480_L1": dict(width=640, height=480, kind="checker", levels=1,
                              max_feats=300, fast_thresh=20, fast_thresh_lo=0, frames=1),
    "kitti_1241x376_L8": dict(width=1241, height=376, kind="planes", levels=8,
                              max_feats=2000, fast_thresh=20, fast_thresh_lo=7, frames=100),
    "euroc_752x480_L8": dict(width=752, height=480, kind="euroc", levels=8,
                             max_feats=1200, fast_thresh=20, fast_thresh_lo=7, frames=200),
    "fhd_1920x1080_L8": dict(width=1920, height=1080, kind="planes", levels=8,
                             max_feats=3000, fast_thresh=20, fast_thresh_lo=7, frames=100),
}

# The mixed multi-stream batch: 4 streams of each size, pyramid depth per size group.
MIXED_STREAMS = (
    [dict(width=640, height=480, kind="checker", levels=4, max_feats=1000)] * 4
    + [dict(width=752, height=480, kind="euroc", levels=5, max_feats=1200)] * 4
    + [dict(width=1241, height=376, kind="planes", levels=6, max_feats=2000)] * 4
    + [dict(width=1920, height=1080, kind="planes", levels=8, max_feats=3000)] * 4
)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _fill_polygons(canvas: np.ndarray, rng: np.random.Generator, count: int,
                   rmin: float, rmax: float) -> None:
    """Paint `count` random star-shaped polygons (3-8 vertices) in place."""
    H, W = canvas.shape
    for _ in range(count):
        nv = int(rng.integers(3, 9))
        cx = rng.uniform(0, W)
        cy = rng.uniform(0, H)
        ang = np.sort(rng.uniform(0, 2 * np.pi, nv))
        rad = rng.uniform(rmin, rmax, nv)
        vx = cx + rad * np.cos(ang)
        vy = cy + rad * np.sin(ang)
        val = float(rng.integers(0, 256))
        x0 = max(int(np.floor(vx.min())), 0); x1 = min(int(np.ceil(vx.max())) + 1, W)
        y0 = max(int(np.floor(vy.min())), 0); y1 = min(int(np.ceil(vy.max())) + 1, H)
        if x0 >= x1 or y0 >= y1:
            continue
        px, py = np.meshgrid(np.arange(x0, x1) + 0.5, np.arange(y0, y1) + 0.5)
        inside = np.zeros(px.shape, bool)
        for i in range(nv):
            ax, ay = vx[i], vy[i]
            bx, by = vx[(i + 1) % nv], vy[(i + 1) % nv]
            cond = (ay > py) != (by > py)
            with np.errstate(divide="ignore", invalid="ignore"):
                xint = ax + (py - ay) * (bx - ax) / (by - ay)
            inside ^= cond & (px < xint)
        canvas[y0:y1, x0:x1][inside] = val


def _blocky_noise(rng: np.random.Generator, H: int, W: int, block: int, amp: float) -> np.ndarray:
    gh, gw = H // block + 2, W // block + 2
    g = rng.uniform(-amp, amp, (gh, gw))
    return np.repeat(np.repeat(g, block, 0), block, 1)[:H, :W]


def _texture(rng: np.random.Generator, H: int, W: int, polys_per_mpx: float) -> np.ndarray:
    t = np.full((H, W), 128.0)
    t += _blocky_noise(rng, H, W, 16, 40.0)
    t += _blocky_noise(rng, H, W, 6, 25.0)
    _fill_polygons(t, rng, max(1, int(polys_per_mpx * H * W / 1e6)), 4.0, 30.0)
    return t


def _finish(img: np.ndarray, rng: np.random.Generator, sigma: float) -> np.ndarray:
    noisy = img + np.round(rng.normal(0.0, sigma, img.shape))
    return np.clip(noisy, 0, 255).astype(np.uint8)


@dataclass
class StereoPair:
    left: np.ndarray
    right: np.ndarray
    disparity: np.ndarray  # ground-truth disparity of each left pixel


def checker_pair(width: int, height: int, seed: int, disparity: int = 16,
                 polygons: int = 150, sigma: float = 2.0) -> StereoPair:
    """Checkerboard + polygons, constant disparity."""
    rng = _rng(seed)
    Wc = width + disparity
    yy, xx = np.mgrid[0:height, 0:Wc]
    canvas = np.where(((xx // 8) + (yy // 8)) % 2 == 0, 64.0, 192.0)
    _fill_polygons(canvas, rng, polygons, 6.0, 60.0)
    left = canvas[:, :width]
    right = canvas[:, disparity:disparity + width]
    d = np.full((height, width), disparity, np.int32)
    return StereoPair(_finish(left, rng, sigma), _finish(right, rng, sigma), d)


@lru_cache(maxsize=8)
def _planes_world(width: int, height: int, world_seed: int, max_disp: int = 96, boxes: int = 20):
    rng = _rng(world_seed)
    margin = max_disp + 64
    Wt = width + margin
    ground = _texture(rng, height, Wt, 600.0)
    far = _texture(rng, height, Wt, 300.0)
    bl = []
    for _ in range(boxes):
        bw = int(rng.integers(width // 20, width // 6))
        bh = int(rng.integers(height // 10, height // 3))
        bx = int(rng.integers(0, max(1, width - bw)))
        by = int(rng.integers(0, max(1, height - bh)))
        bd = int(rng.integers(8, max_disp + 1))
        bl.append((bx, by, bw, bh, bd, _texture(rng, bh, bw + margin, 900.0)))
    bl.sort(key=lambda b: b[4])  # far to near
    return ground, far, bl


def planes_pair(width: int, height: int, frame: int, world_seed: int, frame_seed: int,
                max_disp: int = 96, sigma: float = 2.0, shift_per_frame: float = 0.5) -> StereoPair:
    """Ground plane (disparity proportional to row) + background + boxes."""
    ground, far, boxes = _planes_world(width, height, world_seed, max_disp)
    rng = _rng(frame_seed)
    t = shift_per_frame * frame
    it = int(np.floor(t)); ft = t - it
    horizon = int(0.35 * height)
    rows = np.arange(height)
    d_row = np.where(rows > horizon,
                     np.round(max_disp * (rows - horizon) / max(1, height - 1 - horizon)), 0).astype(np.int64)

    def sample(tex, xs, ys):
        xs = xs + it
        a = tex[ys, np.clip(xs, 0, tex.shape[1] - 1)]
        b = tex[ys, np.clip(xs + 1, 0, tex.shape[1] - 1)]
        return (1.0 - ft) * a + ft * b

    xs = np.arange(width)[None, :].repeat(height, 0)
    ys = rows[:, None].repeat(width, 1)
    base_tex = np.where(ys > horizon, 1, 0)

    def render(view_shift_sign):
        # view_shift_sign 0: left view; 1: right view (looks up x + d)
        dmap = d_row[:, None].repeat(width, 1).astype(np.int64)
        lx = xs + view_shift_sign * dmap
        img = np.where(base_tex == 1, sample(ground, lx, ys), sample(far, xs, ys))
        dist = np.where(base_tex == 1, dmap, 0)
        for (bx, by, bw, bh, bd, tex) in boxes:
            # columns of this view that see the box (left x in [bx, bx + bw))
            c0 = max(bx - view_shift_sign * bd, 0)
            c1 = min(bx + bw - view_shift_sign * bd, width)
            r0, r1 = by, min(by + bh, height)
            if c0 >= c1 or r0 >= r1:
                continue
            sub_x = xs[r0:r1, c0:c1] + view_shift_sign * bd - bx
            sub_y = ys[r0:r1, c0:c1] - by
            img[r0:r1, c0:c1] = sample(tex, np.clip(sub_x, 0, tex.shape[1] - 2), sub_y)
            dist[r0:r1, c0:c1] = bd
        return img, dist

    left, dl = render(0)
    right, _ = render(1)
    return StereoPair(_finish(left, rng, sigma), _finish(right, rng, sigma), dl.astype(np.int32))


def euroc_pair(width: int, height: int, frame: int, world_seed: int, frame_seed: int) -> StereoPair:
    """Planes scene with low-texture regions, motion blur and gain jumps."""
    base = planes_pair(width, height, frame, world_seed, frame_seed, max_disp=64, sigma=0.0)
    wrng = _rng(world_seed + 7)
    low = np.zeros((height, width), bool)
    target = 0.30 * width * height
    while low.sum() < target:
        rw = int(wrng.integers(width // 10, width // 3)); rh = int(wrng.integers(height // 10, height // 3))
        rx = int(wrng.integers(0, width - rw)); ry = int(wrng.integers(0, height - rh))
        low[ry:ry + rh, rx:rx + rw] = True
    level = float(wrng.integers(60, 200))
    frng = _rng(frame_seed + 1_000_000)
    blur_len = int(frng.integers(5, 16))
    gain_rng = _rng(world_seed + 13 + frame // 25)
    gain = 1.0 + float(gain_rng.choice([-0.2, 0.0, 0.2]))
    out = []
    for img in (base.left, base.right):
        f = img.astype(np.float64)
        smooth = level + frng.normal(0.0, 3.0, f.shape)
        f = np.where(low, smooth, f)
        k = np.ones(blur_len) / blur_len
        pad = np.pad(f, ((0, 0), (blur_len // 2, blur_len - 1 - blur_len // 2)), mode="edge")
        cs = np.cumsum(pad, axis=1)
        cs = np.concatenate([np.zeros((height, 1)), cs], axis=1)
        f = (cs[:, blur_len:] - cs[:, :-blur_len]) * k[0]
        f = f * gain
        out.append(_finish(f, frng, 2.0))
    return StereoPair(out[0], out[1], base.disparity)


def stereo_pair(kind: str, width: int, height: int, frame: int = 0, stream: int = 0,
                config_id: int = 0) -> StereoPair:
    """One seeded stereo pair.  Seeds: world = 1000*config_id + 500 + stream,
    frame noise = 1000*config_id + frame + 100000*stream."""
    world_seed = 1000 * config_id + 500 + stream
    frame_seed = 1000 * config_id + frame + 100000 * stream
    if kind == "checker":
        return checker_pair(width, height, frame_seed)
    if kind == "planes":
        return planes_pair(width, height, frame, world_seed, frame_seed)
    if kind == "euroc":
        return euroc_pair(width, height, frame, world_seed, frame_seed)
    raise ValueError(f"unknown scene kind {kind!r}")


def workload_pair(name: str, frame: int = 0) -> StereoPair:
    w = WORKLOADS[name]
    cfg_id = list(WORKLOADS).index(name) + 1
    return stereo_pair(w["kind"], w["width"], w["height"], frame, 0, cfg_id)


def random_image(height: int, width: int, seed: int, kind: str = "polygons") -> np.ndarray:
    """Small seeded test image (polygons over blocky noise)."""
    rng = _rng(seed)
    t = _texture(rng, height, width, 2000.0)
    return _finish(t, rng, 2.0)


@dataclass
class CornerScene:
    image: np.ndarray     # uint8 [H, W]
    corners: np.ndarray   # float64 [N, 2]: (x, y) of every polygon vertex; pixel (i, j) covers [i, i+1) x [j, j+1)


def corner_polygons(width: int, height: int, seed: int, polygons: int = 14, rmin: float = 10.0,
                    rmax: float = 24.0, margin: float = 24.0):
    """Labeled shapes for the repeatability study of Bounded Rectification:
    convex polygons inscribed in circles (3-6 vertices, every interior angle
    in [30, 150] degrees), pairwise 6 px apart, inside the disc about the
    image centre that keeps them `margin` px from every edge under any
    rotation; background and fills at least 40 grey levels apart.
    Returns (background, [(vertices [nv, 2], fill, (cx, cy, r)), ...])."""
    rng = _rng(seed)
    cx, cy = width / 2.0, height / 2.0
    reach = min(width, height) / 2.0 - rmax - margin
    bg = float(rng.integers(80, 177))
    shapes = []
    tries = 0
    while len(shapes) < polygons and tries < 20000:
        tries += 1
        r = rng.uniform(rmin, rmax)
        rho, th = reach * np.sqrt(rng.uniform()), rng.uniform(0, 2 * np.pi)
        px, py = cx + rho * np.cos(th), cy + rho * np.sin(th)
        if any(np.hypot(px - qx, py - qy) < r + qr + 6.0 for _, _, (qx, qy, qr) in shapes):
            continue
        nv = int(rng.integers(3, 7))
        phi = np.sort(rng.uniform(0, 2 * np.pi, nv))
        gaps = np.diff(np.concatenate([phi, phi[:1] + 2 * np.pi]))
        # inscribed polygon: the interior angle at vertex i is pi - (gap before + gap after) / 2
        interior = np.pi - (gaps + np.roll(gaps, 1)) / 2.0
        if interior.min() < np.radians(30) or interior.max() > np.radians(150):
            continue
        fill = float(rng.integers(0, 256))
        if abs(fill - bg) < 40:
            continue
        verts = np.stack([px + r * np.cos(phi), py + r * np.sin(phi)], axis=1)
        shapes.append((verts, fill, (px, py, r)))
    return bg, shapes


def corner_scene(width: int, height: int, angle_deg: float, seed: int, polygons: int = 14,
                 supersample: int = 4, sigma: float = 2.0, dots: int = 0) -> CornerScene:
    """The shapes of corner_polygons(seed) rotated by angle_deg about the image
    centre (counter-clockwise on screen, y down), rendered with area
    coverage from supersample^2 samples per pixel, plus Gaussian noise of
    sigma (seeded by the seed and the angle).  `dots` unlabeled discs of
    radius 1-2 px (contrast >= 40, 6 px clear of the polygons' circles,
    rotating with the scene) stand in for the specks and blobs of real
    images, which are not corners."""
    bg, shapes = corner_polygons(width, height, seed, polygons)
    cx, cy = width / 2.0, height / 2.0
    items = [(v, f, True) for v, f, _ in shapes]
    if dots:
        drng = _rng(seed * 7919 + 17)
        reach = min(width, height) / 2.0 - 30.0
        placed = 0
        while placed < dots:
            rho, th = reach * np.sqrt(drng.uniform()), drng.uniform(0, 2 * np.pi)
            px, py = cx + rho * np.cos(th), cy + rho * np.sin(th)
            rd = drng.uniform(1.0, 2.0)
            if any(np.hypot(px - qx, py - qy) < qr + rd + 6.0 for _, _, (qx, qy, qr) in shapes):
                continue
            fill = float(drng.integers(0, 256))
            if abs(fill - bg) < 40:
                continue
            k = np.arange(16) * (2 * np.pi / 16)
            items.append((np.stack([px + rd * np.cos(k), py + rd * np.sin(k)], axis=1), fill, False))
            placed += 1
    a = np.radians(angle_deg)
    ca, sa = np.cos(a), np.sin(a)
    img = np.full((height, width), bg)
    corners = []
    ss = supersample
    for verts, fill, labeled in items:
        dx, dy = verts[:, 0] - cx, verts[:, 1] - cy
        v = np.stack([cx + ca * dx + sa * dy, cy - sa * dx + ca * dy], axis=1)
        if labeled:
            corners.append(v)
        x0, x1 = int(np.floor(v[:, 0].min())), int(np.ceil(v[:, 0].max())) + 1
        y0, y1 = int(np.floor(v[:, 1].min())), int(np.ceil(v[:, 1].max())) + 1
        sx = x0 + (np.arange((x1 - x0) * ss) + 0.5) / ss
        sy = y0 + (np.arange((y1 - y0) * ss) + 0.5) / ss
        px, py = np.meshgrid(sx, sy)
        inside = np.ones(px.shape, bool)
        nv = len(v)
        area2 = sum(v[i, 0] * v[(i + 1) % nv, 1] - v[(i + 1) % nv, 0] * v[i, 1] for i in range(nv))
        for i in range(nv):  # convex: inside every edge's half-plane (orientation from the signed area)
            ax, ay = v[i]
            bx, by = v[(i + 1) % nv]
            cross = (bx - ax) * (py - ay) - (by - ay) * (px - ax)
            inside &= cross * np.sign(area2) >= 0
        cov = inside.reshape(y1 - y0, ss, x1 - x0, ss).mean(axis=(1, 3))
        img[y0:y1, x0:x1] = img[y0:y1, x0:x1] * (1 - cov) + fill * cov
    rng = _rng(seed * 1000003 + int(round((angle_deg % 360.0) * 1000)))
    return CornerScene(_finish(img, rng, sigma), np.concatenate(corners) if corners else np.zeros((0, 2)))
