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


def test_algorithmic_ops_per_pixel():
    """Eq. 1-3 in scalar form: 16 differences, 2 x 16 labels, 2 x 16 mask bits
    and 3 for the table test per pixel; 31 + 1 more per corner (response and
    cell maximum)."""
    assert bench.alg_ops_per_pixel(0.0) == 83
    assert bench.alg_ops_per_pixel(0.5) == pytest.approx(83 + 16)
    assert "83" in bench.ALG_OPS_DEFINITION


def test_code_hash_ignores_comments_and_whitespace(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) {\n  return x + 1; // one\n}\n/* block */\n")
    b.write_text("int f(int x)   {   return x + 1; }\n// other comment\n")
    assert bench.code_hash(str(a)) == bench.code_hash(str(b))
    b.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_hash(str(a)) != bench.code_hash(str(b))


def test_emitted_line_carries_the_contract(monkeypatch, capsys):
    """Our arm's JSON line, emitted on the CPU from synthetic stage times with
    the committed ncu summaries: every contract key, the integer-issue
    roofline of the dominant stage with its instruction count and DRAM
    traffic taken from the summary, the HBM view beside it, and the launch
    count of the timed mode."""
    import json
    import types
    import bench
    monkeypatch.setattr(bench, "alu_peak", lambda dev: (40.3e12, 152, 2070.0))
    args = types.SimpleNamespace(steps=50, warmup=3, workload="kitti_1241x376_L8", mode="graph_streams8",
                                 no_cpu_baseline=True)
    pairs, params, lo = bench.make_workload(args.workload, 2)
    stage = {"pyramid": 0.774, "skip": 0.0, "detect": 0.865, "pfa_nms": 0.048, "pfa_final": 0.066, "orb": 0.259,
             "match": 0.172}
    clocks = types.SimpleNamespace(summary=lambda: {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []})
    e2e = {"value": 43000.0, "unit": bench.UNIT, "h2d_bytes_per_step": 1, "d2h_bytes_per_step": 1}
    bench.emit(args, 1, len(pairs), 47800.0, 2.09 * 50, {"graph_streams8": 47800.0},
               {k: v * 50 for k, v in stage.items()}, [2000] * 4, pairs, params, lo, e2e, clocks, (128, 128, 0, 0, 0),
               None, 0)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
                "gpu_launches"):
        assert key in line, key
    assert line["config"]["workload"].startswith("kitti_1241x376_L8")
    assert line["gpu_launches"] == 8 * bench.LAUNCHES_PER_CALL * 50
    roof = line["roofline"]
    prof = bench.profile_summary("k_fast_bits", "kitti_1241x376_L8")
    assert prof is not None and roof["bound"] == "alu" and roof["kernel"] == "k_fast_bits"
    lane_ops = bench.profile_number(prof, "inst_executed_warp_per_launch") * 32
    assert roof["inst_per_launch"] == lane_ops
    assert abs(roof["achieved"] - lane_ops / 0.865e-3) < 1e-6 * roof["achieved"]
    assert abs(roof["frac"] - roof["achieved"] / 40.3e12) < 1e-12
    assert roof["traffic"] == bench.profile_number(prof, "dram_bytes_per_launch_full_workload")
    assert roof["hbm"]["algorithmic_bytes_per_launch"] == bench.algorithmic_bytes("detect", pairs, params, [1])
    assert line["path_hbm"]["frac"] > 0 and line["cpu_baseline"] is None
    assert line["path_hbm"]["by_mode"]["graph_streams8"]["frac"] == line["path_hbm"]["frac"]
    assert line["config"]["tuning"] == {"nms_kernel": 0, "detect_ctas_per_sm": 0, "tile_order": 0, "source": "--tile"}


def test_results_table_covers_every_config(capsys):
    """The committed bench lines under results/ hold all five workloads, each
    a contract line with every mode's throughput and its whole-path HBM share,
    and the table generator prints a row for each."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_table", os.path.join(ROOT, "results", "make_table.py"))
    mt = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mt)
    rows = mt.load()
    assert [w for w, _ in rows] == mt.ORDER
    for w, d in rows:
        assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["n_gpus"] == 1
        assert d["value"] > 0 and d["clocks"]["sm_mhz"] and not set(d["clocks"]["reasons"]) & {
            "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
        for m in ("graph_streams8", "batched", "plain", "learned_skip"):
            assert d["modes"][m] > 0 and d["path_hbm"]["by_mode"][m]["frac"] > 0, (w, m)
        # the end-to-end line: every route timed, the headline is the first route's figure,
        # and both directions' bytes are counted
        e = d["e2e"]
        assert set(e["routes"]) == {r[0] for r in bench.E2E_ROUTES} | {"single_context"}, w
        assert e["value"] == e["routes"][bench.E2E_ROUTES[0][0]] and e["unit"] == bench.UNIT
        assert e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    mt.main()
    out = capsys.readouterr().out
    assert all(f"| {w} " in out for w in mt.ORDER)
