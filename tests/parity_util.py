"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare it element by element with the oracle."""
import numpy as np

ANGLE_TOL = 1e-4  # radians: float atan2 on the GPU vs double atan2 in the oracle

EXACT_FIELDS = ("x", "y", "X", "Y", "level", "response", "k_levels", "k_resp", "angle_bin", "desc")


def params_from(oracle, **kw):
    p = oracle.FrontendParams()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def frontend_for(J, p, max_width=1920, max_height=1080, max_pairs=16, max_feats=None, stream=None):
    return J.Frontend(device=0, stream=stream, max_width=max_width, max_height=max_height, max_levels=8,
                      max_feats=max_feats or max(p.max_feats, 4000), max_pairs=max_pairs,
                      fast_thresh_lo=p.fast_thresh_lo, p_min=p.p_min, p_max=p.p_max,
                      k_per_cell=p.k_per_cell, nms_q=p.nms_q, border=p.border, max_disp=p.max_disp,
                      row_band_px=p.row_band_px, match_max_dist=p.match_max_dist, pfa_rule=p.pfa_rule,
                      response_mode=p.response_mode, pyramid_mode=p.pyramid_mode)


def gpu_pair(J, fe, left, right, p, host=False):
    import torch
    if host:
        l, r = np.ascontiguousarray(left), np.ascontiguousarray(right)
    else:
        l = torch.from_numpy(np.ascontiguousarray(left)).cuda()
        r = torch.from_numpy(np.ascontiguousarray(right)).cuda()
    fe.extract(l, r, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    fe.sync()
    kl = J.to_numpy(fe.keypoints(0, 0))
    kr = J.to_numpy(fe.keypoints(0, 1))
    m = J.to_numpy(fe.matches(0))
    return kl, kr, m


def compare_keypoints(got, want, what=""):
    n = want["count"]
    assert got["count"] == n, f"{what}: count {got['count']} != oracle {n}"
    for f in EXACT_FIELDS:
        g = np.asarray(got[f])[:n]
        w = np.asarray(want[f])[:n]
        if not np.array_equal(g, w):
            bad = np.nonzero((g != w).reshape(n, -1).any(axis=1))[0]
            i = int(bad[0])
            raise AssertionError(f"{what}: field {f} differs at {len(bad)} keypoints; first {i}: "
                                 f"gpu {g[i]} oracle {w[i]} (level {want['level'][i]}, x {want['x'][i]}, "
                                 f"y {want['y'][i]})")
    da = np.abs(np.asarray(got["angle"])[:n].astype(np.float64) - np.asarray(want["angle"])[:n].astype(np.float64))
    da = np.minimum(da, 2 * np.pi - da)
    assert n == 0 or da.max() <= ANGLE_TOL, f"{what}: angle error {da.max()}"


def compare_matches(got, want_tuple, what=""):
    idx, disp, dist = want_tuple
    n = len(idx)
    assert got["count"] == n
    assert np.array_equal(got["right_idx"][:n], idx), f"{what}: right_idx"
    assert np.array_equal(got["disparity"][:n], disp), f"{what}: disparity"
    assert np.array_equal(got["dist"][:n], dist), f"{what}: dist"
