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
