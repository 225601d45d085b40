"""The C-ABI library loads and exports every symbol of include/jslam.h, and
its host-built tables (no device work) equal the oracle's, which derives
them again from the same written definitions."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def jslam():
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam as J
    return J


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "jslam.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(jslam_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(jslam):
    declared = _declared_functions()
    assert len(declared) >= 15
    lib = jslam.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(jslam.SYMBOLS) == declared


def test_status_strings(jslam):
    for s in (0, -1, -2, -3, -4, -5, -6):
        assert jslam.status_str(s)


def test_pattern_table_matches_oracle(jslam, oracle):
    assert np.array_equal(jslam.pattern_table(), oracle.pattern_rotated())


@pytest.mark.parametrize("W0,H0,levels,cell", [(1241, 376, 8, 32), (752, 480, 8, 32), (1920, 1080, 8, 32),
                                               (640, 480, 1, 32), (203, 157, 3, 7), (333, 290, 5, 15)])
def test_geometry_projection_band_match_oracle(jslam, oracle, W0, H0, levels, cell):
    w, h, c = jslam.level_geometry(W0, H0, levels, 1.2, cell)
    ow, oh, oc = oracle.level_geometry(W0, H0, levels, 1.2, cell)
    assert np.array_equal(w, ow) and np.array_equal(h, oh) and np.array_equal(c, oc)
    for n in range(levels):
        for v in range(0, int(w[n]), 3):
            assert jslam.project(v, n, 1.2, W0) == oracle.project(v, n, 1.2, W0)
        for v in range(0, int(h[n]), 3):
            assert jslam.project(v, n, 1.2, H0) == oracle.project(v, n, 1.2, H0)
        assert jslam.match_band(n, 1.2, 2) == oracle.match_band(n, 1.2, 2)


def test_other_scales(jslam, oracle):
    for scale in (1.1, 1.25, 1.5, 2.0):
        w, h, c = jslam.level_geometry(999, 777, 6, scale, 40)
        ow, oh, oc = oracle.level_geometry(999, 777, 6, scale, 40)
        assert np.array_equal(w, ow) and np.array_equal(h, oh) and np.array_equal(c, oc)


@pytest.mark.parametrize("p_min,p_max", [(9, 13), (9, 16), (12, 14), (1, 16), (16, 16)])
def test_corner_table_matches_oracle(jslam, oracle, p_min, p_max):
    table = jslam.corner_table(p_min, p_max)
    bits = np.unpackbits(table.view(np.uint8), bitorder="little").astype(bool)
    want = np.array([p_min <= oracle.longest_run(m) <= p_max for m in range(1 << 16)])
    assert np.array_equal(bits, want)


def test_cardinal_pretest_is_necessary(oracle):
    """The detection kernel rejects a pixel early when, for both polarities,
    (F0 | F8) & (F4 | F12) fails on its ring flags.  That is only sound if
    every mask whose longest circular run is 8 or more passes it, and the
    kernel uses it only for P_min >= 8; 7 is too short."""
    runs = np.array([oracle.longest_run(m) for m in range(1 << 16)])
    m = np.arange(1 << 16)
    f = lambda q: (m >> q) & 1
    passes = ((f(0) | f(8)) & (f(4) | f(12))).astype(bool)
    assert passes[runs >= 8].all()
    assert not passes[runs == 7].all()


def test_bitsliced_run_window_identity(oracle):
    """The bit-sliced detection kernel decides Eq. 3 for run bounds [9, 13]
    by windows of flags: A3_q = F_q F_q+1 F_q+2, a run of 9 at q is
    A3_q A3_q+3 A3_q+6, a run of 14 is that and A3_q+9 A3_q+11, and the
    pixel is a corner when some run of 9 exists and no run of 14 does.  Over
    all 2^16 ring masks this equals 9 <= longest circular run <= 13."""
    m = np.arange(1 << 16)
    F = [(m >> q) & 1 for q in range(16)]
    A3 = [F[q] & F[(q + 1) % 16] & F[(q + 2) % 16] for q in range(16)]
    r9 = np.zeros_like(m)
    r14 = np.zeros_like(m)
    for q in range(16):
        a9 = A3[q] & A3[(q + 3) % 16] & A3[(q + 6) % 16]
        r9 |= a9
        r14 |= a9 & A3[(q + 9) % 16] & A3[(q + 11) % 16]
    got = (r9 & (1 - r14)).astype(bool)
    want = np.array([9 <= oracle.longest_run(int(v)) <= 13 for v in m])
    assert np.array_equal(got, want)


def test_bitplane_transpose_identity():
    """The detection kernel's bit-plane transpose (three delta swaps per 8x8
    bit block, then byte permutes gathering byte i of the four blocks into
    word i) gives word i, bit j = bit i of byte j, for random 32-byte chunks
    (the same word operations in numpy)."""
    rng = np.random.default_rng(7)
    by = rng.integers(0, 256, (4096, 32), dtype=np.uint64)
    w = [(by[:, 4 * k] | by[:, 4 * k + 1] << 8 | by[:, 4 * k + 2] << 16 | by[:, 4 * k + 3] << 24) for k in range(8)]
    M = np.uint64(0xFFFFFFFF)
    for blk in range(4):
        lo, hi = w[2 * blk], w[2 * blk + 1]
        for sh, mask in ((7, 0x00AA00AA), (14, 0x0000CCCC)):
            t = (lo ^ (lo >> np.uint64(sh))) & np.uint64(mask); lo = lo ^ t ^ ((t << np.uint64(sh)) & M)
            t = (hi ^ (hi >> np.uint64(sh))) & np.uint64(mask); hi = hi ^ t ^ ((t << np.uint64(sh)) & M)
        t = (lo ^ ((hi << np.uint64(4)) & M)) & np.uint64(0xF0F0F0F0)
        w[2 * blk], w[2 * blk + 1] = lo ^ t, hi ^ (t >> np.uint64(4))
    byte = lambda x, i: (x >> np.uint64(8 * i)) & np.uint64(0xFF)
    for i in range(8):
        half, bi = divmod(i, 4)
        got = byte(w[half], bi) | byte(w[2 + half], bi) << np.uint64(8) | \
            byte(w[4 + half], bi) << np.uint64(16) | byte(w[6 + half], bi) << np.uint64(24)
        want = np.zeros(len(by), np.uint64)
        for j in range(32):
            want |= ((by[:, j] >> np.uint64(i)) & np.uint64(1)) << np.uint64(j)
        assert np.array_equal(got, want), i


def test_sector_float_margin_agrees_with_double(jslam):
    """The orientation kernel decides each sector boundary in float when
    |m01 cos - m10 sin| exceeds (|m01| + |m10|) 2^-20 and in IEEE double
    otherwise.  Emulated here with numpy float32 / float64 (both round to
    nearest, no fused operations) on random moments and on moments placed
    next to every boundary: where float decides, it agrees with double."""
    b = np.arange(30)
    phi = 2 * np.pi * b / 30.0
    c64, s64 = np.cos(phi), np.sin(phi)  # the argument holds for any table with |c|, |s| <= 1
    c32, s32 = c64.astype(np.float32), s64.astype(np.float32)
    rng = np.random.default_rng(0)
    a = rng.integers(-(1 << 22), 1 << 22, 200000)
    bb = rng.integers(-(1 << 22), 1 << 22, 200000)
    # moments almost exactly along a boundary direction
    k = rng.integers(0, 30, 200000)
    r = rng.integers(1, 1 << 22, 200000).astype(np.float64)
    a2 = np.round(r * s64[k]).astype(np.int64) + rng.integers(-2, 3, 200000)
    b2 = np.round(r * c64[k]).astype(np.int64) + rng.integers(-2, 3, 200000)
    m01 = np.concatenate([a, a2]); m10 = np.concatenate([bb, b2])
    decided = fallback = 0
    for j in range(30):
        t64 = (m01 * c64[j]) - (m10 * s64[j])
        fa, fb = m01.astype(np.float32), m10.astype(np.float32)
        t32 = (fa * c32[j]).astype(np.float32) - (fb * s32[j]).astype(np.float32)
        margin = (np.abs(fa) + np.abs(fb)) * np.float32(2.0 ** -20)
        sure = np.abs(t32) > margin
        assert np.array_equal((t32 > 0)[sure], (t64 >= 0)[sure])
        decided += int(sure.sum()); fallback += int((~sure).sum())
    assert fallback > 0 and decided > 10 * fallback  # half the samples sit on boundaries on purpose
