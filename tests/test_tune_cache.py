"""The autotuner's persistent cache (host code only, no GPU): batch keys that
tell GPUs, configurations and batches apart, and a JSON file that keeps every
pick, survives rewrites and treats a damaged file as empty."""
import json

import numpy as np
import pytest


@pytest.fixture(scope="module")
def J():
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


def _jobs(J, sizes, **kw):
    return [J.Job(np.zeros((h, w), np.uint8), np.zeros((h, w), np.uint8), **kw) for w, h in sizes]


def test_keys_tell_batches_apart(J):
    base = J.tune_key("NVIDIA GB300", 152, {}, _jobs(J, [(1241, 376)] * 2))
    assert base == J.tune_key("NVIDIA GB300", 152, {}, _jobs(J, [(1241, 376)] * 2))  # deterministic
    others = [J.tune_key("NVIDIA B200", 148, {}, _jobs(J, [(1241, 376)] * 2)),
              J.tune_key("NVIDIA GB300", 144, {}, _jobs(J, [(1241, 376)] * 2)),
              J.tune_key("NVIDIA GB300", 152, {"k_per_cell": 2}, _jobs(J, [(1241, 376)] * 2)),
              J.tune_key("NVIDIA GB300", 152, {"fast_thresh_lo": 7}, _jobs(J, [(1241, 376)] * 2)),
              J.tune_key("NVIDIA GB300", 152, {}, _jobs(J, [(1241, 376)] * 3)),
              J.tune_key("NVIDIA GB300", 152, {}, _jobs(J, [(1242, 376)] * 2)),
              J.tune_key("NVIDIA GB300", 152, {}, _jobs(J, [(1241, 376)] * 2, levels=7)),
              J.tune_key("NVIDIA GB300", 152, {}, _jobs(J, [(1241, 376)] * 2, scale=1.25)),
              J.tune_key("NVIDIA GB300", 152, {}, _jobs(J, [(1241, 376)] * 2, max_feats=1000))]
    assert len(set(others + [base])) == len(others) + 1
    assert '"' not in J.tune_key('GPU "x"\\', 1, {}, _jobs(J, [(64, 64)]))


def test_key_buffer_too_small(J):
    import ctypes as C
    cfg = J.Config()
    J.lib().jslam_default_config(C.byref(cfg))
    pb = J.PreparedBatch(_jobs(J, [(640, 480)]))
    buf = C.create_string_buffer(16)
    assert J.lib().jslam_tune_key(b"NVIDIA GB300", 152, C.byref(cfg), pb.array, pb.n, buf, 16) == J.ERR_CAPACITY


def test_store_and_find(J, tmp_path):
    path = str(tmp_path / "tune.json")
    assert J.tune_cache_get(path, "a") is None  # no file yet
    J.tune_cache_put(path, "a", (128, 128, 0, 0, 0), 0.86)
    J.tune_cache_put(path, "b|jobs=640x480", (64, 64, 1, 2, 1), 0.5)
    assert J.tune_cache_get(path, "a") == (128, 128, 0, 0, 0)
    assert J.tune_cache_get(path, "b|jobs=640x480") == (64, 64, 1, 2, 1)
    assert J.tune_cache_get(path, "c") is None
    J.tune_cache_put(path, "a", (128, 32, 0, 3, 1), 0.7)  # replace
    assert J.tune_cache_get(path, "a") == (128, 32, 0, 3, 1)
    doc = json.load(open(path))  # plain JSON, readable by other tools
    assert doc["format"] == "jslam-tune-cache" and doc["version"] == 1
    assert doc["entries"]["a"] == {"tile_w_px": 128, "tile_h_px": 32, "nms_kernel": 0, "detect_ctas_per_sm": 3,
                                   "tile_order": 1, "stage_ms": pytest.approx(0.7)}
    assert set(doc["entries"]) == {"a", "b|jobs=640x480"}


def test_damaged_or_foreign_files(J, tmp_path):
    path = tmp_path / "tune.json"
    for text in ("", "{", "not json", '{"entries": {"a": {"tile_w_px": }}}', '{"entries": {"a\\u0041": {}}}'):
        path.write_text(text)
        assert J.tune_cache_get(str(path), "a") is None
    path.write_text('{"entries": {"a": {"tile_w_px": 4, "tile_h_px": 64}}}')  # out-of-range pick
    assert J.tune_cache_get(str(path), "a") is None
    # extra fields and other top-level keys are tolerated; an entry without
    # the tile order (written before it existed) reads as order 0
    path.write_text('{"note": {"x": "y"}, "entries": {"a": {"tile_w_px": 96, "tile_h_px": 16, "nms_kernel": 1, '
                    '"detect_ctas_per_sm": 0, "stage_ms": 1.5, "by": "hand"}}, "version": 1}')
    assert J.tune_cache_get(str(path), "a") == (96, 16, 1, 0, 0)
    path.write_text("garbage")
    J.tune_cache_put(str(path), "k", (128, 64, 0, 0))  # a damaged file is rewritten
    assert json.load(open(path))["entries"] == {"k": {"tile_w_px": 128, "tile_h_px": 64, "nms_kernel": 0,
                                                       "detect_ctas_per_sm": 0, "tile_order": 0, "stage_ms": 0.0}}


def test_refuses_invalid_entries(J, tmp_path):
    path = str(tmp_path / "tune.json")
    for bad in ((130, 64, 0, 0), (126, 64, 0, 0), (128, 4, 0, 0), (128, 64, 2, 0), (128, 64, 0, 9),
                (128, 64, 0, 0, 2), (128, 64, 0, 0, -1)):
        with pytest.raises(J.JslamError) as e:
            J.tune_cache_put(path, "a", bad)
        assert e.value.status == J.ERR_ARG
    with pytest.raises(J.JslamError):
        J.tune_cache_put(path, 'a"b', (128, 64, 0, 0))
    with pytest.raises(J.JslamError):
        J.tune_cache_put(str(tmp_path / "missing_dir" / "t.json"), "a", (128, 64, 0, 0))
