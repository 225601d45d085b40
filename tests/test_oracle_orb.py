"""Pins of the oracle's orientation (intensity centroid), angle bins, BRIEF
pattern and descriptor (Sec. III, streamlined extraction with ORB)."""
import math

import numpy as np
import pytest

from conftest import read_golden

R = 15


def test_splitmix64_published_vector(oracle):
    want = [int(r[0], 16) for r in read_golden("splitmix64_seed0.txt")]
    assert oracle.splitmix64(0, 3) == want


def test_std_normal_moments(oracle):
    z = oracle.std_normals(12345, 200000)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.015
    assert abs((np.abs(z) < 1.0).mean() - 0.6827) < 0.005  # Gaussian mass within 1 sigma


def test_pattern_properties(oracle):
    p = oracle.pattern_base().astype(int)
    assert p.shape == (256, 4)
    assert np.all(p[:, 0] ** 2 + p[:, 1] ** 2 <= 169)
    assert np.all(p[:, 2] ** 2 + p[:, 3] ** 2 <= 169)
    assert not np.any((p[:, 0] == p[:, 2]) & (p[:, 1] == p[:, 3]))
    # only p = q is redrawn: pairs sharing one coordinate remain (each
    # coordinate is shared by about 1 / (2 sqrt(pi) sigma) = 4.5 % of pairs)
    assert ((p[:, 0] == p[:, 2]) & (p[:, 1] != p[:, 3])).sum() >= 4
    assert ((p[:, 1] == p[:, 3]) & (p[:, 0] != p[:, 2])).sum() >= 4
    # isotropic Gaussian with sigma 31/5, truncated to the radius-13 disk
    assert 4.5 < p.std() < 6.2
    assert abs(p.mean()) < 0.6
    assert len({tuple(r) for r in p.tolist()}) > 250


def test_pattern_spread_matches_the_truncated_lattice_gaussian(oracle):
    """Each point is (lround(sigma g1), lround(sigma g2)) for independent
    standard normals, kept when inside the radius-13 disk: the lattice point
    (i, j) has probability proportional to the Gaussian mass of its unit
    square, restricted to i^2 + j^2 <= 169.  The sample mean of the 1024
    squared coordinates lies within 3 standard errors of that distribution's
    E[x^2] (27.9 for sigma = 31/5; a sigma of 31/4 would give 32.6)."""
    from scipy.stats import norm
    sigma = 31.0 / 5.0
    i = np.arange(-13, 14)
    m1 = norm.cdf((i + 0.5) / sigma) - norm.cdf((i - 0.5) / sigma)
    I, J = np.meshgrid(i, i, indexing="ij")
    P = np.outer(m1, m1) * (I ** 2 + J ** 2 <= 169)
    P /= P.sum()
    ex2, ex4 = (P * I ** 2).sum(), (P * I ** 4).sum()
    se = np.sqrt((ex4 - ex2 ** 2) / 1024)
    p = oracle.pattern_base().astype(float)
    assert abs((p ** 2).mean() - ex2) < 3 * se, ((p ** 2).mean(), ex2, se)


def test_rotated_pattern(oracle):
    base = oracle.pattern_base().astype(float)
    rot = oracle.pattern_rotated().astype(float)
    assert np.array_equal(rot[0], base)
    for b in range(30):
        phi = 2 * math.pi * b / 30
        c, s = math.cos(phi), math.sin(phi)
        for pt in (0, 2):
            x, y = base[:, pt], base[:, pt + 1]
            xr, yr = c * x - s * y, s * x + c * y
            assert np.all(np.abs(rot[b][:, pt] - xr) <= 0.5 + 1e-9)
            assert np.all(np.abs(rot[b][:, pt + 1] - yr) <= 0.5 + 1e-9)
            assert np.all(rot[b][:, pt] ** 2 + rot[b][:, pt + 1] ** 2 <= 15 ** 2)


def _ramp(alpha, size=41, g=3.0, base=128.0):
    c = size // 2
    yy, xx = np.mgrid[0:size, 0:size] - c
    img = base + g * (xx * math.cos(alpha) + yy * math.sin(alpha))
    return np.clip(np.round(img), 0, 255).astype(np.uint8), c


def _bin_of(theta):
    t = theta % (2 * math.pi)
    return int(t // (2 * math.pi / 30)) % 30


@pytest.mark.parametrize("deg", [0, 13, 45, 90, 137, 180, 200, 271, 359, -30])
def test_orientation_of_ramp(oracle, deg):
    alpha = math.radians(deg)
    img, c = _ramp(alpha)
    m10, m01, theta, b = oracle.orient(img, c, c)
    # centroid of a linear ramp over a disk points along its gradient
    d = math.atan2(math.sin(theta - alpha), math.cos(theta - alpha))
    assert abs(d) < 0.02
    want = _bin_of(theta)
    edge = (theta % (2 * math.pi)) / (2 * math.pi / 30)
    if abs(edge - round(edge)) > 1e-6:
        assert b == want


def test_sector_boundaries_are_half_open(oracle):
    """Sector b covers [phi_b, phi_b+1): a centroid exactly on a boundary is in
    the sector that starts there.  Ramps along the axes give m01 = 0 (or
    m10 = 0) exactly, by symmetry: 0 deg is on phi_0 and 180 deg on phi_15,
    while 90 and 270 deg lie inside sectors 7 and 22."""
    for deg, want in ((0, 0), (180, 15), (90, 7), (270, 22)):
        img, c = _ramp(math.radians(deg))
        m10, m01, theta, b = oracle.orient(img, c, c)
        assert (m01 == 0 and m10 != 0) if deg in (0, 180) else (m10 == 0 and m01 != 0)
        assert b == want, (deg, b)


def test_orientation_moments_brute_force(oracle):
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (41, 41)).astype(np.uint8)
    m10, m01, theta, b = oracle.orient(img, 20, 20)
    yy, xx = np.mgrid[-R:R + 1, -R:R + 1]
    disk = xx ** 2 + yy ** 2 <= R * R
    patch = img[20 - R:21 + R, 20 - R:21 + R].astype(np.int64)
    assert m10 == int((xx * patch)[disk].sum())
    assert m01 == int((yy * patch)[disk].sum())
    assert abs(theta - math.atan2(m01, m10)) < 1e-12
    assert b == _bin_of(theta)


def test_symmetric_blob_has_zero_angle(oracle):
    yy, xx = np.mgrid[-20:21, -20:21]
    img = np.clip(200 - (xx ** 2 + yy ** 2) / 3, 0, 255).astype(np.uint8)
    m10, m01, theta, b = oracle.orient(img, 20, 20)
    assert (m10, m01, theta, b) == (0, 0, 0.0, 0)


def test_descriptor_constant_patch_is_zero(oracle):
    rot = oracle.pattern_rotated()
    img = np.full((41, 41), 90, np.uint8)
    for b in (0, 7, 29):
        assert not oracle.describe(img, 20, 20, rot[b]).any()


def test_descriptor_of_ramp(oracle):
    """On I = a + g x the bit of pair i is [p'_x < q'_x]; fixes the pair
    orientation, the bit order and the word packing."""
    rot = oracle.pattern_rotated()
    xx = np.arange(41)[None, :].repeat(41, 0)
    img = (40 + 4 * xx).astype(np.uint8)
    for b in (0, 5, 17):
        d = oracle.describe(img, 20, 20, rot[b])
        bits = (rot[b][:, 0].astype(int) < rot[b][:, 2].astype(int))
        want = np.zeros(8, np.uint32)
        for i in np.nonzero(bits)[0]:
            want[i // 32] |= np.uint32(1) << np.uint32(i % 32)
        assert np.array_equal(d, want)


def test_descriptor_swap_flips_bits(oracle):
    rng = np.random.default_rng(0)
    img = rng.permutation(np.arange(41 * 41) % 256).reshape(41, 41).astype(np.uint8)
    rot = oracle.pattern_rotated()
    for b in (0, 11):
        tab = rot[b]
        vals_p = img[20 + tab[:, 1].astype(int), 20 + tab[:, 0].astype(int)]
        vals_q = img[20 + tab[:, 3].astype(int), 20 + tab[:, 2].astype(int)]
        tie_free = vals_p != vals_q
        swapped = tab[:, [2, 3, 0, 1]].copy()
        d1 = oracle.describe(img, 20, 20, tab)
        d2 = oracle.describe(img, 20, 20, swapped)
        bits1 = np.unpackbits(d1.view(np.uint8), bitorder="little")
        bits2 = np.unpackbits(d2.view(np.uint8), bitorder="little")
        assert np.all(bits1[tie_free] != bits2[tie_free])
        assert np.all(bits1[~tie_free] == 0) and np.all(bits2[~tie_free] == 0)
