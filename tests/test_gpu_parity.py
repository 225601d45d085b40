"""Parity of the CUDA path (through the C ABI) with the oracle: bit-exact
keypoints, scores, sectors, descriptors and matches, angles within 1e-4 rad.
Sizes span several tiles with ragged edges; the full workload shapes are
compared in full (the oracle finishes them in seconds)."""
import dataclasses

import numpy as np
import pytest

from paper_2410_04090_gb300 import scenes
from parity_util import compare_keypoints, compare_matches, frontend_for, gpu_pair, params_from

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def J():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_04090_gb300 import build
    build.build()
    from paper_2410_04090_gb300 import jslam
    return jslam


def _check_pair(J, oracle, left, right, p, host=False, fe=None):
    own = fe is None
    fe = fe or frontend_for(J, p)
    try:
        kl, kr, m = gpu_pair(J, fe, left, right, p, host=host)
    finally:
        if own:
            fe.close()
    ol, orr, om = oracle.extract_pair(left, right, p)
    compare_keypoints(kl, ol, "left")
    compare_keypoints(kr, orr, "right")
    compare_matches(m, om, "matches")
    return ol, orr, om


def test_small_ragged_multilevel(J, oracle):
    pair = scenes.planes_pair(203, 157, 0, 31, 32)
    p = params_from(oracle, levels=3, max_feats=500, cell=16)
    ol, _, _ = _check_pair(J, oracle, pair.left, pair.right, p)
    assert ol["count"] > 20


def test_pyramid_levels_match_oracle(J, oracle):
    import torch
    pair = scenes.planes_pair(317, 251, 0, 5, 6)
    p = params_from(oracle, levels=6, max_feats=1000)
    fe = frontend_for(J, p)
    l = torch.from_numpy(pair.left).cuda(); r = torch.from_numpy(pair.right).cuda()
    fe.extract(l, r, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.sync()
    for side, img in ((0, pair.left), (1, pair.right)):
        for n in range(p.levels):
            lv = fe.level(0, side, n)
            raw = lv["raw"].cpu().numpy()
            want = img if n == 0 else oracle.pyramid_level(img, p.scale, n)
            assert np.array_equal(raw, want), (side, n)
            assert np.array_equal(lv["blurred"].cpu().numpy(), oracle.blur(want)), (side, n)
    fe.close()


@pytest.mark.parametrize("name", ["single_640x480_L1", "kitti_1241x376_L8", "euroc_752x480_L8"])
def test_workload_parity(J, oracle, name):
    w = scenes.WORKLOADS[name]
    pair = scenes.workload_pair(name, 1)
    p = params_from(oracle, levels=w["levels"], max_feats=w["max_feats"], fast_thresh=w["fast_thresh"],
                    fast_thresh_lo=w["fast_thresh_lo"])
    ol, orr, om = _check_pair(J, oracle, pair.left, pair.right, p)
    assert ol["count"] > 100 and (om[0] >= 0).sum() > 50


def test_full_hd_parity(J, oracle):
    w = scenes.WORKLOADS["fhd_1920x1080_L8"]
    pair = scenes.workload_pair("fhd_1920x1080_L8", 0)
    p = params_from(oracle, levels=8, max_feats=w["max_feats"], fast_thresh_lo=7)
    _check_pair(J, oracle, pair.left, pair.right, p)


def test_host_memory_input(J, oracle):
    pair = scenes.workload_pair("kitti_1241x376_L8", 2)
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=7)
    _check_pair(J, oracle, pair.left, pair.right, p, host=True)


def test_strided_device_input(J, oracle):
    import torch
    pair = scenes.planes_pair(300, 200, 0, 41, 42)
    p = params_from(oracle, levels=4, max_feats=400)
    fe = frontend_for(J, p)
    big_l = torch.zeros((200, 384), dtype=torch.uint8, device="cuda")
    big_r = torch.zeros((200, 384), dtype=torch.uint8, device="cuda")
    big_l[:, :300] = torch.from_numpy(pair.left).cuda()
    big_r[:, :300] = torch.from_numpy(pair.right).cuda()
    fe.extract(big_l[:, :300], big_r[:, :300], p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.match(); fe.sync()
    from paper_2410_04090_gb300 import jslam
    ol, orr, om = oracle.extract_pair(pair.left, pair.right, p)
    compare_keypoints(jslam.to_numpy(fe.keypoints(0, 0)), ol, "left")
    compare_matches(jslam.to_numpy(fe.matches(0)), om)
    fe.close()


@pytest.mark.parametrize("kw", [
    dict(k_per_cell=3),
    dict(nms_q=5),
    dict(nms_q=1),
    dict(pfa_rule=1),
    dict(p_max=16),            # classic FAST (Eq. 2) as the unbounded special case
    dict(p_min=12, p_max=14),
    dict(p_min=8, p_max=13),   # shortest arc the cardinal pre-test covers
    dict(p_min=6, p_max=10),   # below it: the pre-test is off
    dict(cell=7),
    dict(cell=100),
    dict(max_feats=5),         # cap binds hard; ties resolved in canonical order
    dict(fast_thresh=8, fast_thresh_lo=3),
    dict(fast_thresh=60, fast_thresh_lo=25),
    dict(border=25),
    dict(scale=1.5, levels=4),
    dict(match_max_dist=30, max_disp=40, row_band_px=0),
])
def test_parameter_variants(J, oracle, kw):
    pair = scenes.planes_pair(420, 300, 0, 77, 78)
    base = dict(levels=5, max_feats=800)
    base.update(kw)
    p = params_from(oracle, **base)
    _check_pair(J, oracle, pair.left, pair.right, p)


def test_wide_segments(J, oracle):
    """Segments (cell rows of a level) of 1248 candidate slots -- k = 8 per
    8 px cell on a 1241-wide image -- in the one-CTA-per-segment NMS kernel
    (batches whose segments have at most 96 slots use one warp per segment)."""
    pair = scenes.planes_pair(1241, 376, 0, 31, 32)
    p = params_from(oracle, levels=2, max_feats=3000, cell=8, k_per_cell=8)
    _check_pair(J, oracle, pair.left, pair.right, p)


@pytest.mark.parametrize("w,h,k", [(640, 480, 1), (1241, 376, 1), (640, 300, 3), (640, 300, 5)])
def test_narrow_segments(J, oracle, w, h, k):
    """Largest segment (cells per row x k) of 22 slots (640 px), 42 (1241 px)
    and 66 (3 per cell on 640 px) -- the warp-per-segment NMS kernel with
    one, two and three slots per lane -- and 110 (5 per cell: the CTA
    kernel)."""
    pair = scenes.planes_pair(w, h, 0, 41, 42)
    p = params_from(oracle, levels=6, max_feats=1500, fast_thresh_lo=7, k_per_cell=k)
    _check_pair(J, oracle, pair.left, pair.right, p)


def test_maximum_image_size(J, oracle):
    """The largest accepted image, 4096 x 4096 with 8 levels and 4000 features:
    keypoints, descriptors and angles against the oracle (one image, used as
    both sides, keeps the oracle's share of the test to one extraction)."""
    import torch
    img = scenes.random_image(4096, 4096, 5)
    p = params_from(oracle, levels=8, max_feats=4000, fast_thresh_lo=7)
    fe = frontend_for(J, p, max_width=4096, max_height=4096, max_pairs=1)
    t = torch.from_numpy(img).cuda()
    fe.extract(t, t, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    fe.sync()
    want = oracle.extract_image(img, p)
    compare_keypoints(J.to_numpy(fe.keypoints(0, 0)), want, "4096 left")
    compare_keypoints(J.to_numpy(fe.keypoints(0, 1)), want, "4096 right")
    m = J.to_numpy(fe.matches(0))
    n = want["count"]
    assert (m["right_idx"][:n] == np.arange(n)).mean() > 0.99  # identical images match themselves
    fe.close()


def test_minimum_size_levels(J, oracle):
    # the deepest level is exactly 2 * border + 1 pixels on its short side
    W0 = H0 = int(np.ceil(39 * 1.2 ** 3))
    p = params_from(oracle, levels=4, max_feats=200, cell=8)
    while not oracle.check_params(W0, H0, p):
        W0 += 1; H0 += 1
    pair = scenes.planes_pair(W0, H0, 0, 3, 4)
    _check_pair(J, oracle, pair.left, pair.right, p)


def test_flat_image_has_no_keypoints(J, oracle):
    flat = np.full((120, 160), 128, np.uint8)
    p = params_from(oracle, levels=2, max_feats=100)
    ol, _, om = _check_pair(J, oracle, flat, flat, p)
    assert ol["count"] == 0 and len(om[0]) == 0


def test_repeated_calls_reuse_buffers(J, oracle):
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=7)
    fe = frontend_for(J, p)
    try:
        for f in (0, 1, 0):
            pair = scenes.workload_pair("kitti_1241x376_L8", f)
            _check_pair(J, oracle, pair.left, pair.right, p, fe=fe)
        # a different shape on the same context, then back
        small = scenes.planes_pair(300, 240, 0, 9, 10)
        _check_pair(J, oracle, small.left, small.right, params_from(oracle, levels=4, max_feats=2000,
                                                                     fast_thresh_lo=7), fe=fe)
        pair = scenes.workload_pair("kitti_1241x376_L8", 3)
        _check_pair(J, oracle, pair.left, pair.right, p, fe=fe)
    finally:
        fe.close()


def test_mixed_batch(J, oracle):
    """Several stereo pairs of different sizes and depths in one launch set."""
    import torch
    specs = [(640, 480, "checker", 4, 1000), (752, 480, "euroc", 5, 1200), (1241, 376, "planes", 6, 2000),
             (500, 300, "planes", 8, 700), (640, 480, "checker", 1, 300)]
    p0 = params_from(oracle, fast_thresh_lo=7)
    fe = frontend_for(J, p0, max_pairs=8)
    jobs, pairs = [], []
    from paper_2410_04090_gb300 import jslam
    for i, (w, h, kind, lv, mf) in enumerate(specs):
        pr = scenes.stereo_pair(kind, w, h, frame=i, stream=i, config_id=4)
        pairs.append((pr, lv, mf))
        jobs.append(jslam.Job(torch.from_numpy(pr.left).cuda(), torch.from_numpy(pr.right).cuda(), lv, 1.2, 20, 32, mf))
    fe.extract_batch(jobs)
    fe.match()
    fe.sync()
    for i, (pr, lv, mf) in enumerate(pairs):
        p = params_from(oracle, levels=lv, max_feats=mf, fast_thresh_lo=7)
        ol, orr, om = oracle.extract_pair(pr.left, pr.right, p)
        compare_keypoints(jslam.to_numpy(fe.keypoints(i, 0)), ol, f"pair {i} left")
        compare_keypoints(jslam.to_numpy(fe.keypoints(i, 1)), orr, f"pair {i} right")
        compare_matches(jslam.to_numpy(fe.matches(i)), om, f"pair {i}")
    fe.close()


def test_download_result_block(J, oracle):
    import torch
    pair = scenes.workload_pair("euroc_752x480_L8", 3)
    p = params_from(oracle, levels=8, max_feats=1200, fast_thresh_lo=7)
    fe = frontend_for(J, p)
    fe.extract(pair.left, pair.right, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    buf = torch.empty(fe.result_bytes(0), dtype=torch.uint8).pin_memory()
    fe.download(0, buf)
    fe.sync()
    ol, orr, om = oracle.extract_pair(pair.left, pair.right, p)
    left = fe.result_view(0, buf, 0)
    compare_keypoints(left, ol, "left")
    compare_keypoints(fe.result_view(0, buf, 1), orr, "right")
    compare_matches({"count": left["count"], "right_idx": left["match_right_idx"],
                     "disparity": left["match_disparity"], "dist": left["match_dist"]}, om)
    fe.close()


def test_host_frames_back_to_back_and_ranged_download(J, oracle):
    """Host frames of two pairs in one buffer (one upload copy), a strided
    host frame (one 2-D copy), and one ranged download of all result
    blocks, each block byte-identical to its single-pair download."""
    import torch
    p = params_from(oracle, levels=5, max_feats=700, fast_thresh_lo=7)
    prs = [scenes.planes_pair(420, 300, k, 90, 91) for k in range(2)] + [scenes.planes_pair(300, 200, 0, 92, 93)]
    flat = np.zeros(4 * 420 * 300, np.uint8)
    views = []
    for k in range(2):
        for j, img in enumerate((prs[k].left, prs[k].right)):
            v = flat[(2 * k + j) * 420 * 300:(2 * k + j + 1) * 420 * 300].reshape(300, 420)
            v[...] = img
            views.append(v)
    wide = np.zeros((200, 512), np.uint8)          # pitch 512 > 384 = 300 rounded up to 128
    wide[:, :300] = prs[2].left
    strided = wide[:, :300]
    fe = frontend_for(J, p, max_pairs=4)
    jobs = [J.Job(views[0], views[1], p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats),
            J.Job(views[2], views[3], p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats),
            J.Job(strided, np.ascontiguousarray(prs[2].right), p.levels, p.scale, p.fast_thresh, p.cell,
                  p.max_feats)]
    fe.extract_batch(jobs)
    fe.match()
    total, offs = fe.result_range(0, 3)
    big = torch.empty(total, dtype=torch.uint8).pin_memory()
    fe.download_range(0, 3, big)
    singles = []
    for k in range(3):
        t = torch.empty(fe.result_bytes(k), dtype=torch.uint8).pin_memory()
        fe.download(k, t)
        singles.append(t)
    fe.sync()
    for k, pr in enumerate(prs):
        ol, orr, om = oracle.extract_pair(pr.left, pr.right, p)
        compare_keypoints(J.to_numpy(fe.keypoints(k, 0)), ol, f"pair {k} left")
        compare_keypoints(J.to_numpy(fe.keypoints(k, 1)), orr, f"pair {k} right")
        compare_matches(J.to_numpy(fe.matches(k)), om, f"pair {k}")
        block = big[offs[k]: offs[k] + singles[k].numel()]
        assert torch.equal(block, singles[k]), k
        compare_keypoints(fe.result_view(k, block.clone(), 0), ol, f"pair {k} ranged view")
    with pytest.raises(J.JslamError):
        fe.download_range(0, 3, torch.empty(total - 1, dtype=torch.uint8).pin_memory())
    with pytest.raises(J.JslamError):
        fe.result_range(2, 2)
    fe.close()


def test_argument_errors(J):
    import torch
    fe = J.Frontend(device=0, max_width=640, max_height=480, max_levels=4, max_feats=500, max_pairs=2)
    img = torch.zeros((100, 120), dtype=torch.uint8, device="cuda")
    bad = [dict(levels=0), dict(levels=5), dict(scale=1.0), dict(fast_thresh=0), dict(fast_thresh=255),
           dict(cell=0), dict(cell=129), dict(max_feats=0), dict(max_feats=501)]
    for kw in bad:
        args = dict(levels=2, scale=1.2, fast_thresh=20, cell=32, max_feats=100)
        args.update(kw)
        with pytest.raises(J.JslamError) as e:
            fe.extract(img, img, **args)
        assert e.value.status == J.ERR_ARG, kw
    tiny = torch.zeros((45, 60), dtype=torch.uint8, device="cuda")  # level 1 is 38 rows < 2 * 19 + 1
    with pytest.raises(J.JslamError) as e:
        fe.extract(tiny, tiny, 2, 1.2, 20, 32, 100)
    assert e.value.status == J.ERR_ARG
    fe.extract(tiny, tiny, 1, 1.2, 20, 32, 100)
    big = torch.zeros((481, 100), dtype=torch.uint8, device="cuda")
    with pytest.raises(J.JslamError):
        fe.extract(big, big, 1, 1.2, 20, 32, 100)
    with pytest.raises(J.JslamError) as e:
        fe.extract(img, img[:, :110], 1, 1.2, 20, 32, 100)  # left/right sizes differ
    assert e.value.status == J.ERR_ARG
    fresh = J.Frontend(device=0)
    with pytest.raises(J.JslamError) as e:
        fresh.match()
    assert e.value.status == J.ERR_STATE
    with pytest.raises(J.JslamError) as e:
        J.Frontend(device=0, p_min=10, p_max=9)
    assert e.value.status == J.ERR_ARG
    # a rejected call leaves the context usable
    fe.extract(img, img, 2, 1.2, 20, 32, 100)
    fe.sync()
    fe.close(); fresh.close()


def test_stage_timing(J, oracle):
    import torch
    pair = scenes.workload_pair("kitti_1241x376_L8", 0)
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=7)
    fe = frontend_for(J, p)
    with pytest.raises(J.JslamError):
        fe.stage_times()
    fe.enable_stage_timing(True)
    l = torch.from_numpy(pair.left).cuda(); r = torch.from_numpy(pair.right).cuda()
    fe.extract(l, r, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    fe.sync()
    t = fe.stage_times()
    assert set(t) == set(J.STAGES) and t["refine"] == 0.0, t      # refinement not run
    assert all(v > 0 for k, v in t.items() if k != "refine"), t
    fe.extract(l, r, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
    fe.match()
    fe.refine_matches(5, 5, 0.0)
    fe.sync()
    t = fe.stage_times()
    assert all(v > 0 for v in t.values()), t
    fe.enable_stage_timing(False)
    fe.close()


def test_shared_torch_streams(J, oracle):
    """The context runs on a stream the caller passes, including torch's
    default stream; events on that stream bracket the library's work."""
    import torch
    pair = scenes.workload_pair("kitti_1241x376_L8", 4)
    p = params_from(oracle, levels=8, max_feats=2000, fast_thresh_lo=7)
    ol, orr, om = oracle.extract_pair(pair.left, pair.right, p)
    from paper_2410_04090_gb300 import jslam
    for stream in (torch.cuda.default_stream(), torch.cuda.Stream()):
        fe = J.Frontend(device=0, stream=stream, max_width=1241, max_height=376, max_feats=2000,
                        fast_thresh_lo=7, max_pairs=1)
        fe.enable_stage_timing(True)
        with torch.cuda.stream(stream):
            l = torch.from_numpy(pair.left).cuda(); r = torch.from_numpy(pair.right).cuda()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fe.extract(l, r, p.levels, p.scale, p.fast_thresh, p.cell, p.max_feats)
            fe.match()
            e1.record(stream)
        e1.synchronize()  # no jslam_sync: the event alone must cover the work
        t = fe.stage_times()
        assert e0.elapsed_time(e1) >= 0.9 * sum(t.values())
        fe.sync()
        compare_keypoints(jslam.to_numpy(fe.keypoints(0, 0)), ol, "left")
        compare_matches(jslam.to_numpy(fe.matches(0)), om)
        fe.close()


@pytest.mark.parametrize("tune", [(32, 8), (64, 128), (128, 128), (128, 32)])
def test_tuning_does_not_change_results(J, oracle, tune):
    pair = scenes.planes_pair(501, 333, 0, 55, 56)
    p = params_from(oracle, levels=6, max_feats=900, fast_thresh_lo=7)
    fe = frontend_for(J, p)
    fe.set_tuning(*tune)
    _check_pair(J, oracle, pair.left, pair.right, p, fe=fe)
    fe.close()


def _mixed_streams(J, specs, frame):
    import torch
    pairs, jobs = [], []
    for i, sp in enumerate(specs):
        pr = scenes.stereo_pair(sp["kind"], sp["width"], sp["height"], frame=frame, stream=i, config_id=4)
        pairs.append(pr)
        jobs.append(J.Job(torch.from_numpy(pr.left).cuda(), torch.from_numpy(pr.right).cuda(), sp["levels"], 1.2, 20,
                          32, sp["max_feats"]))
    return pairs, jobs


def _check_batch(J, oracle, fe, pairs, specs):
    for i, (pr, sp) in enumerate(zip(pairs, specs)):
        p = params_from(oracle, levels=sp["levels"], max_feats=sp["max_feats"], fast_thresh_lo=7)
        ol, orr, om = oracle.extract_pair(pr.left, pr.right, p)
        compare_keypoints(J.to_numpy(fe.keypoints(i, 0)), ol, f"pair {i} left")
        compare_keypoints(J.to_numpy(fe.keypoints(i, 1)), orr, f"pair {i} right")
        compare_matches(J.to_numpy(fe.matches(i)), om, f"pair {i}")


def test_graph_replay_on_new_device_frames(J, oracle):
    """jslam_graph_launch_jobs: the captured graph replayed on new device
    frames (new tensors, not the captured buffers), two replays in flight
    before one sync, each followed by a download of its results; then the
    refusals: another batch shape, a host image, a rebuilt plan."""
    import torch
    specs = scenes.MIXED_STREAMS[::4]  # one stream of each size
    fe = frontend_for(J, params_from(oracle, fast_thresh_lo=7), max_pairs=4, stream=torch.cuda.Stream())
    _, jobs0 = _mixed_streams(J, specs, 0)
    fe.graph_capture(jobs0)
    frames = {f: _mixed_streams(J, specs, f) for f in (1, 2)}
    torch.cuda.synchronize()  # the uploads (torch's stream) land before the context's stream reads them
    total, offs = fe.result_range(0, len(specs))
    blocks = {}
    for f, (_, jobs) in frames.items():  # no sync between the replays
        fe.graph_launch(jobs)
        blocks[f] = torch.empty(total, dtype=torch.uint8).pin_memory()
        fe.download_range(0, len(specs), blocks[f])
    fe.sync()
    _check_batch(J, oracle, fe, frames[2][0], specs)  # device views: the last replay
    for f, (pairs, _) in frames.items():
        for i, (pr, sp) in enumerate(zip(pairs, specs)):
            p = params_from(oracle, levels=sp["levels"], max_feats=sp["max_feats"], fast_thresh_lo=7)
            ol, orr, om = oracle.extract_pair(pr.left, pr.right, p)
            blk = blocks[f][offs[i]:].clone()
            compare_keypoints(fe.result_view(i, blk, 0), ol, f"frame {f} pair {i} left")
            compare_keypoints(fe.result_view(i, blk, 1), orr, f"frame {f} pair {i} right")
    # refusals
    _, jobs1 = frames[1]
    with pytest.raises(J.JslamError) as e:
        fe.graph_launch(jobs1[:3])  # fewer pairs
    assert e.value.status == J.ERR_ARG
    other = list(jobs1)
    other[0] = J.Job(other[0].left, other[0].right, other[0].levels - 1, 1.2, 20, 32, other[0].max_feats)
    with pytest.raises(J.JslamError) as e:
        fe.graph_launch(other)  # another depth
    assert e.value.status == J.ERR_ARG
    host = list(jobs1)
    host[1] = J.Job(other[1].left.cpu().numpy(), other[1].right, other[1].levels, 1.2, 20, 32, other[1].max_feats)
    with pytest.raises(J.JslamError) as e:
        fe.graph_launch(host)  # a host image
    assert e.value.status == J.ERR_ARG
    fe.extract_batch(jobs1[:2])  # another batch shape rebuilds the plan: the graph is stale
    with pytest.raises(J.JslamError) as e:
        fe.graph_launch()
    assert e.value.status == J.ERR_STATE
    with pytest.raises(J.JslamError) as e:
        fe.graph_launch(jobs1)
    assert e.value.status == J.ERR_STATE
    fe.sync()
    fe.close()


def _batch_outputs(J, fe, n):
    return [(J.to_numpy(fe.keypoints(i, 0)), J.to_numpy(fe.keypoints(i, 1)), J.to_numpy(fe.matches(i)))
            for i in range(n)]


def test_every_tuning_gives_identical_results(J, oracle):
    """Every launch shape the tuner can pick -- detection tile, persistent
    CTAs per SM, NMS kernel, tile order -- gives the same keypoints,
    descriptors and matches, bit for bit (the default's equal the
    oracle's)."""
    import torch
    specs = scenes.MIXED_STREAMS[::4]
    fe = frontend_for(J, params_from(oracle, fast_thresh_lo=7), max_pairs=4)
    pairs, jobs = _mixed_streams(J, specs, 0)
    torch.cuda.synchronize()
    fe.extract_batch(jobs); fe.match(); fe.sync()
    _check_batch(J, oracle, fe, pairs, specs)
    ref = _batch_outputs(J, fe, len(specs))
    for tw, th in ((128, 64), (128, 32), (128, 128), (64, 64), (64, 128), (96, 48)):
        for nms in (0, 1):
            for ctas, order in ((0, 0), (1, 0), (2, 0), (0, 1), (2, 1)):
                fe.set_tuning(tw, th, nms, ctas, order)
                fe.extract_batch(jobs); fe.match(); fe.sync()
                for i, (a, b) in enumerate(zip(ref, _batch_outputs(J, fe, len(specs)))):
                    what = f"tile {tw}x{th} nms {nms} ctas {ctas} order {order} pair {i}"
                    for side in (0, 1):
                        assert a[side]["count"] == b[side]["count"], what
                        for f in ("x", "y", "X", "Y", "level", "response", "k_levels", "k_resp", "angle_bin",
                                  "desc", "angle"):
                            assert np.array_equal(a[side][f], b[side][f]), (what, side, f)
                    for f in ("right_idx", "disparity", "dist"):
                        assert np.array_equal(a[2][f], b[2][f]), (what, f)
    fe.close()


def test_autotune_cache_hits_on_a_new_context(J, oracle, tmp_path):
    import json
    import torch
    specs = scenes.MIXED_STREAMS[::4]
    pairs, jobs = _mixed_streams(J, specs, 0)
    torch.cuda.synchronize()
    path = str(tmp_path / "tune.json")
    fe = frontend_for(J, params_from(oracle, fast_thresh_lo=7), max_pairs=4)
    pick = fe.autotune(jobs, cache=path)
    assert fe.last_tune_hit is False
    entries = json.load(open(path))["entries"]
    assert len(entries) == 1 and list(entries.values())[0]["stage_ms"] > 0
    fe.close()
    fe2 = frontend_for(J, params_from(oracle, fast_thresh_lo=7), max_pairs=4)
    assert fe2.autotune(jobs, cache=path) == pick and fe2.last_tune_hit is True
    fe2.extract_batch(jobs); fe2.match(); fe2.sync()
    _check_batch(J, oracle, fe2, pairs, specs)
    fe2.close()
    fe3 = frontend_for(J, params_from(oracle, fast_thresh_lo=7, k_per_cell=2), max_pairs=4)
    fe3.autotune(jobs, cache=path)  # another configuration: a miss, a second entry
    assert fe3.last_tune_hit is False and len(json.load(open(path))["entries"]) == 2
    fe3.close()


def test_mixed_sixteen_streams(J, oracle):
    """The mixed multi-stream batch: 4 streams each of 640x480 (4 levels),
    752x480 (5), 1241x376 (6) and 1920x1080 (8), autotuned, in one launch set."""
    specs = scenes.MIXED_STREAMS
    fe = frontend_for(J, params_from(oracle, fast_thresh_lo=7), max_pairs=16)
    pairs, jobs = _mixed_streams(J, specs, 0)
    tile = fe.autotune(jobs)
    assert tile[0] in (64, 128) and tile[1] in (32, 64, 128) and tile[2] in (0, 1) and 0 <= tile[3] <= 8
    assert tile[4] in (0, 1)
    fe.extract_batch(jobs)
    fe.match()
    fe.sync()
    _check_batch(J, oracle, fe, pairs, specs)
    fe.close()


def test_graph_replay_follows_new_frames(J, oracle):
    import torch
    specs = scenes.MIXED_STREAMS[::4]  # one stream of each size
    fe = frontend_for(J, params_from(oracle, fast_thresh_lo=7), max_pairs=4, stream=torch.cuda.Stream())
    pairs, jobs = _mixed_streams(J, specs, 0)
    fe.graph_capture(jobs)
    for frame in (1, 2):
        nxt, _ = _mixed_streams(J, specs, frame)
        for j, pr in zip(jobs, nxt):  # new frames into the captured buffers
            j.left.copy_(torch.from_numpy(pr.left))
            j.right.copy_(torch.from_numpy(pr.right))
        torch.cuda.synchronize()
        fe.graph_launch()
        fe.sync()
        _check_batch(J, oracle, fe, nxt, specs)
    fe.close()


def test_graph_replay_copies_host_frames(J, oracle):
    """A graph captured on pinned host frames that lie back to back in one
    buffer (so their upload is one copy, a node of the graph) copies them
    again on every replay: new frames written into the same host buffer
    between replays give the new frames' keypoints and matches, and the
    ranged download enqueued after each replay holds them too."""
    import torch
    specs = scenes.MIXED_STREAMS[::4]  # one stream of each size
    n = len(specs)
    fe = frontend_for(J, params_from(oracle, fast_thresh_lo=7), max_pairs=4, stream=torch.cuda.Stream())
    frames = {f: [scenes.stereo_pair(sp["kind"], sp["width"], sp["height"], frame=f, stream=i, config_id=4)
                  for i, sp in enumerate(specs)] for f in (0, 1, 2)}
    total = sum(2 * sp["width"] * sp["height"] for sp in specs)
    flat = torch.empty(total, dtype=torch.uint8).pin_memory()
    buf, views, off = flat.numpy(), [], 0
    for sp in specs:
        pv = []
        for _ in range(2):
            pv.append(buf[off: off + sp["width"] * sp["height"]].reshape(sp["height"], sp["width"]))
            off += sp["width"] * sp["height"]
        views.append(pv)

    def fill(pairs):
        for (vl, vr), pr in zip(views, pairs):
            vl[...] = pr.left
            vr[...] = pr.right

    fill(frames[0])
    jobs = [J.Job(vl, vr, sp["levels"], 1.2, 20, 32, sp["max_feats"]) for (vl, vr), sp in zip(views, specs)]
    fe.graph_capture(jobs)
    fe.sync()
    total_b, offs = fe.result_range(0, n)
    for f in (1, 2):
        fill(frames[f])
        fe.graph_launch()
        block = torch.empty(total_b, dtype=torch.uint8).pin_memory()
        fe.download_range(0, n, block)
        fe.sync()
        _check_batch(J, oracle, fe, frames[f], specs)
        for i, (pr, sp) in enumerate(zip(frames[f], specs)):
            p = params_from(oracle, levels=sp["levels"], max_feats=sp["max_feats"], fast_thresh_lo=7)
            ol, orr, om = oracle.extract_pair(pr.left, pr.right, p)
            blk = block[offs[i]:].clone()
            compare_keypoints(fe.result_view(i, blk, 1), orr, f"frame {f} pair {i} right (downloaded)")
    fe.close()


def test_largest_batch_equals_pairs_alone(J, oracle):
    """The largest batch a context accepts (128 pairs, 256 images: the limit
    of the by-value input table) of pairs of nine sizes, depths 1..6, two
    scene kinds and two thresholds: every pair's keypoints, descriptors and
    matches equal those of the same pair extracted alone, bit for bit, and
    four sampled pairs equal the oracle's.  Two pairs have flat images (no
    keypoints on either side, or on the right side only)."""
    import torch
    sizes = [(96, 64), (160, 120), (203, 157), (256, 96), (128, 200), (333, 111), (64, 64), (300, 180), (177, 143)]
    pairs, jobs, ps = [], [], []
    for i in range(128):
        w, h = sizes[i % len(sizes)]
        pr = scenes.stereo_pair("planes" if i % 3 else "euroc", w, h, frame=i, stream=i % 5, config_id=7)
        if i in (50, 51):  # flat frames: no keypoints on both sides (50) or on the right (51)
            flat = np.full((h, w), 128, np.uint8)
            pr = dataclasses.replace(pr, left=flat if i == 50 else pr.left, right=flat)
        p = params_from(oracle, levels=1 + i % 6, max_feats=150 + 7 * i, fast_thresh=20 if i % 4 else 12,
                        fast_thresh_lo=7, cell=16 if i % 2 else 32)
        while p.levels > 1:  # the deepest level must still hold a pixel inside the border
            W, H, _ = oracle.level_geometry(w, h, p.levels, p.scale, p.cell)
            if min(W[-1], H[-1]) >= 2 * p.border + 1:
                break
            p.levels -= 1
        pairs.append(pr)
        ps.append(p)
        jobs.append(J.Job(torch.from_numpy(pr.left).cuda(), torch.from_numpy(pr.right).cuda(), p.levels, p.scale,
                          p.fast_thresh, p.cell, p.max_feats))
    torch.cuda.synchronize()
    base = params_from(oracle, fast_thresh_lo=7)
    fe = frontend_for(J, base, max_width=333, max_height=200, max_pairs=128, max_feats=1100)
    fe.extract_batch(jobs)
    fe.match()
    fe.sync()
    batch = [(J.to_numpy(fe.keypoints(i, 0)), J.to_numpy(fe.keypoints(i, 1)), J.to_numpy(fe.matches(i)))
             for i in range(128)]
    one = frontend_for(J, base, max_width=333, max_height=200, max_pairs=1, max_feats=1100)
    for i, (pr, p) in enumerate(zip(pairs, ps)):
        got = gpu_pair(J, one, pr.left, pr.right, p)
        for side in (0, 1):
            assert batch[i][side]["count"] == got[side]["count"], (i, side)
            for f in ("x", "y", "X", "Y", "level", "response", "k_levels", "k_resp", "angle_bin", "desc", "angle"):
                assert np.array_equal(batch[i][side][f], got[side][f]), (i, side, f)
        for f in ("right_idx", "disparity", "dist"):
            assert np.array_equal(batch[i][2][f], got[2][f]), (i, f)
    assert batch[50][0]["count"] == 0 and batch[51][1]["count"] == 0 and batch[51][0]["count"] > 0
    for i in (0, 51, 67, 127):
        ol, orr, om = oracle.extract_pair(pairs[i].left, pairs[i].right, ps[i])
        compare_keypoints(batch[i][0], ol, f"pair {i} left")
        compare_keypoints(batch[i][1], orr, f"pair {i} right")
        compare_matches(batch[i][2], om, f"pair {i}")
    one.close()
    fe.close()
