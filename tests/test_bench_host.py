"""Host arithmetic of bench.py that needs no GPU: level pixel counts, the
whole path's algorithmic bytes, and the code hash that ties an ncu summary
to the kernel source it was taken from (a summary whose source changed is
not used)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Pair:
    def __init__(self, w, h):
        self.left = np.zeros((h, w), np.uint8)


def test_level_pixels_match_the_multiplier():
    """S_L = sum of zeta^(-2n): the level pixel sum of 1241x376 at 8 levels is
    A0 S_8 up to the rounding of each level's size."""
    px = bench.level_pixels(1241, 376, 8, 1.2)
    assert len(px) == 8 and px[0] == 1241 * 376
    S8 = sum(1.2 ** (-2 * n) for n in range(8))
    assert abs(sum(px) / (1241 * 376) - S8) < 0.01


def test_path_bytes_per_pair():
    """A0 (1 + (S_L - 1) + S_L) + 48 N_kp per image: 5.97 MB per KITTI-shaped
    pair with 2000 keypoints per image."""
    px = bench.level_pixels(1241, 376, 8, 1.2)
    A = sum(px)
    want = 2 * (px[0] + (A - px[0]) + A + 48 * 2000)
    got = bench.path_bytes_per_pair([_Pair(1241, 376)], [dict(levels=8, scale=1.2)], [2000, 2000])
    assert got == want
    assert abs(got / 1e6 - 5.97) < 0.01
    # averaged per pair; keypoints counted per image
    two = bench.path_bytes_per_pair([_Pair(1241, 376), _Pair(752, 480)],
                                    [dict(levels=8, scale=1.2), dict(levels=8, scale=1.2)], [2000, 1000, 1200, 1200])
    p2 = bench.level_pixels(752, 480, 8, 1.2)
    A2 = sum(p2)
    assert two == pytest.approx((want - 48 * 1000 + 2 * (p2[0] + (A2 - p2[0]) + A2) + 48 * 2400) / 2)


def test_code_hash_ignores_comments_and_whitespace(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) {\n  return x + 1; // one\n}\n/* block */\n")
    b.write_text("int f(int x)   {   return x + 1; }\n// other comment\n")
    assert bench.code_hash(str(a)) == bench.code_hash(str(b))
    b.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_hash(str(a)) != bench.code_hash(str(b))
