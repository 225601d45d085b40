#!/usr/bin/env python3
"""Markdown tables of the committed bench lines (results/bench_<workload>.json,
one JSON line each, as `python bench.py --workload <w> --steps 30` printed
them on a GB300): stereo pairs/s of every mode, the whole path's share of
the measured HBM bandwidth per mode, the detection kernel's roofline and the
CPU oracle, as two markdown tables."""
import glob
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
ORDER = ["single_640x480_L1", "kitti_1241x376_L8", "euroc_752x480_L8", "fhd_1920x1080_L8", "mixed16"]
MODES = ["graph_streams8", "graph_streams4", "batched", "graph", "plain", "plain_graph", "learned_skip"]


def load():
    lines = {}
    for path in glob.glob(os.path.join(HERE, "bench_*.json")):
        d = json.loads(open(path).read().strip().splitlines()[-1])
        lines[d["config"]["workload"].split(":")[0]] = d
    return [(w, lines[w]) for w in ORDER if w in lines]


def fmt(v, nd=0):
    return "—" if v is None else f"{v:,.{nd}f}".replace(",", " ")


def e2e_cell(e):
    r = e.get("routes")
    if not r:  # a line from before the graph routes: the extract route and one context
        return f"— / — / — / {fmt(e.get('value'))} ({fmt(e.get('single_context_value'))})"
    return (f"{fmt(r.get('graph_parts4'))} / {fmt(r.get('graph_parts8'))} / {fmt(r.get('graph'))} / "
            f"{fmt(r.get('extract'))} ({fmt(r.get('single_context'))})")


def main():
    rows = load()
    print("| Workload (pairs per step) | " + " | ".join(MODES) + " | e2e: graph_parts4 / graph_parts8 / graph / extract (1 ctx) | CPU oracle, cores (1 core) |")
    print("|---" * (len(MODES) + 3) + "|")
    for w, d in rows:
        m = d["modes"]
        e = d.get("e2e") or {}
        c = d.get("cpu_baseline") or {}
        one = (c.get("single_core") or {}).get("value")
        print(f"| {w} ({d['config']['pairs_per_step']}) | " + " | ".join(fmt(m.get(k)) for k in MODES) +
              f" | {e2e_cell(e)} | "
              f"{fmt(c.get('value'), 2)}, {c.get('cores', '—')} ({fmt(one, 2)}) |")
    print()
    print("| Workload | path HBM: " + " | ".join(MODES) + " | detect ms | detect roofline | clocks MHz |")
    print("|---" * (len(MODES) + 4) + "|")
    for w, d in rows:
        bm = d["path_hbm"].get("by_mode", {})
        r = d.get("roofline") or {}
        st = (r.get("stage_ms_per_launch") or {}).get("detect")
        roof = f"{r.get('bound')} {r.get('frac', 0):.3f}" if r else "—"
        print(f"| {w} | " + " | ".join(f"{100 * bm[k]['frac']:.2f} %" if k in bm else "—" for k in MODES) +
              f" | {fmt(st, 3)} | {roof} | {d['clocks'].get('sm_mhz')} |")


if __name__ == "__main__":
    main()
