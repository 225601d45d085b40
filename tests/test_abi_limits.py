"""jslam_create checks every documented configuration limit before its first
device call: one past each bound it returns JSLAM_ERR_ARG on any machine;
at the bound it passes validation -- on a machine without a GPU the next
step, finding the device, then fails with JSLAM_ERR_CUDA."""
import ctypes

import pytest

from paper_2410_04090_gb300 import jslam

PAST = [dict(max_pairs=0), dict(max_pairs=129), dict(max_width=0), dict(max_width=4097), dict(max_height=4097),
        dict(max_levels=0), dict(max_levels=9), dict(max_feats=0), dict(max_feats=(1 << 20) + 1),
        dict(fast_thresh_lo=255), dict(p_min=0), dict(p_max=17), dict(p_min=14, p_max=13), dict(k_per_cell=0),
        dict(k_per_cell=9), dict(nms_q=0), dict(nms_q=2), dict(nms_q=9), dict(border=15), dict(border=513),
        dict(max_disp=-1), dict(max_disp=4097), dict(row_band_px=-1), dict(row_band_px=65),
        dict(match_max_dist=-1), dict(pfa_rule=-1), dict(pfa_rule=2), dict(response_mode=-1),
        dict(response_mode=2), dict(pyramid_mode=-1), dict(pyramid_mode=2)]
AT = [dict(max_pairs=1), dict(max_pairs=128), dict(max_width=4096, max_height=4096), dict(max_levels=8),
      dict(max_feats=1 << 20), dict(fast_thresh_lo=254), dict(p_min=1, p_max=16), dict(k_per_cell=8),
      dict(nms_q=1), dict(nms_q=7), dict(border=16), dict(border=512), dict(max_disp=0), dict(max_disp=4096),
      dict(row_band_px=64), dict(match_max_dist=0), dict(pfa_rule=1), dict(response_mode=1),
      dict(pyramid_mode=1)]


def _create(**kw):
    L = jslam.lib()
    cfg = jslam.Config()
    L.jslam_default_config(ctypes.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    h = ctypes.c_void_p()
    st = L.jslam_create(ctypes.byref(h), ctypes.byref(cfg))
    if st == jslam.OK:
        L.jslam_destroy(h)
    return st


def test_one_past_each_limit_is_rejected():
    for kw in PAST:
        assert _create(**kw) == jslam.ERR_ARG, kw


def test_each_limit_itself_passes_validation():
    if _create() != jslam.ERR_CUDA:
        pytest.skip("a GPU is present: the bound cases would allocate device memory")
    for kw in AT:
        assert _create(**kw) == jslam.ERR_CUDA, kw
