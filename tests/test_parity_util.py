"""The GPU parity tests' comparators reject every single planted difference
(one descriptor bit, one coordinate or score, the count, an angle just past
the tolerance, one match field) and accept an exact copy with angle jitter
inside the tolerance -- so that "equal to the oracle" in those tests means
what it says.  Runs on the CPU: the planted results are copies of an oracle
extraction."""
import copy

import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import ANGLE_TOL, EXACT_FIELDS, compare_keypoints, compare_matches, params_from


@pytest.fixture(scope="module")
def ref(oracle):
    pair = scenes.planes_pair(320, 240, 0, 5, 6)
    p = params_from(oracle, levels=3, max_feats=400)
    kl, kr, m = oracle.extract_pair(pair.left, pair.right, p)
    assert kl["count"] > 50
    return kl, m


def _as_gpu(kp):
    """The oracle's keypoints laid out like the CUDA path's views: arrays at
    capacity (longer than the count), zero beyond it."""
    got = {"count": kp["count"]}
    for f in EXACT_FIELDS + ("angle",):
        a = np.asarray(kp[f])
        pad = np.zeros((7,) + a.shape[1:], a.dtype)
        got[f] = np.concatenate([a, pad])
    return got


def test_exact_copy_with_angle_jitter_passes(ref):
    kl, _ = ref
    got = _as_gpu(kl)
    rng = np.random.default_rng(0)
    n = kl["count"]
    got["angle"][:n] = (got["angle"][:n] + rng.uniform(-0.9, 0.9, n) * ANGLE_TOL).astype(np.float32)
    compare_keypoints(got, kl)


@pytest.mark.parametrize("field", EXACT_FIELDS)
def test_one_changed_value_fails(ref, field):
    kl, _ = ref
    got = _as_gpu(kl)
    i = kl["count"] // 2
    a = got[field]
    if field == "desc":
        a[i, 5] ^= np.uint32(1 << 17)  # one bit of one descriptor
    else:
        a[i] = a[i] + 1
    with pytest.raises(AssertionError):
        compare_keypoints(got, kl)


def test_count_and_angle_fail(ref):
    kl, _ = ref
    got = _as_gpu(kl)
    got["count"] -= 1
    with pytest.raises(AssertionError):
        compare_keypoints(got, kl)
    got = _as_gpu(kl)
    got["angle"][kl["count"] - 1] += np.float32(2 * ANGLE_TOL)
    with pytest.raises(AssertionError):
        compare_keypoints(got, kl)


def test_angles_compare_across_the_wrap(ref):
    kl, _ = ref
    want = copy.deepcopy(kl)
    want["angle"][0] = np.float32(np.pi - 2e-5)
    got = _as_gpu(want)
    got["angle"][0] = np.float32(-np.pi + 2e-5)  # 4e-5 apart on the circle
    compare_keypoints(got, want)


def test_match_fields_fail(ref):
    _, (idx, disp, dist) = ref
    n = len(idx)
    base = {"count": n, "right_idx": np.concatenate([idx, [-1] * 5]).astype(np.int32),
            "disparity": np.concatenate([disp, [0] * 5]).astype(np.int16),
            "dist": np.concatenate([dist, [0] * 5]).astype(np.uint16)}
    compare_matches(base, (idx, disp, dist))
    for f in ("right_idx", "disparity", "dist"):
        got = copy.deepcopy(base)
        got[f][n // 3] += 1
        with pytest.raises(AssertionError):
            compare_matches(got, (idx, disp, dist))
    got = copy.deepcopy(base)
    got["count"] = n - 1
    with pytest.raises(AssertionError):
        compare_matches(got, (idx, disp, dist))


def test_smoke_comparison_accepts_the_oracle_and_rejects_a_change(oracle):
    """The comparison smoke() applies on the GPU: an oracle result passes it
    (angles compared on the circle), a one-bit change does not."""
    import __graft_entry__ as G
    pair = scenes.planes_pair(320, 240, 0, 11, 12)
    p = params_from(oracle, levels=4, max_feats=400, fast_thresh_lo=7)
    ol, orr, _ = oracle.extract_pair(pair.left, pair.right, p)
    for want in (ol, orr):
        got = _as_gpu(want)
        G._same_keypoints(got, want, "copy")
        wrapped = copy.deepcopy(want)
        wrapped["angle"][0] = np.float32(np.pi - 2e-5)
        g2 = _as_gpu(wrapped)
        g2["angle"][0] = np.float32(-np.pi + 2e-5)   # 4e-5 apart on the circle
        G._same_keypoints(g2, wrapped, "wrap")
        got["desc"][want["count"] - 1, 0] ^= np.uint32(1)
        with pytest.raises(AssertionError):
            G._same_keypoints(got, want, "changed")
