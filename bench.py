#!/usr/bin/env python3
"""Throughput of the stereo frontend hot path on GB300: stereo pairs/s.

One step = the whole hot path (pyramid + Gaussian filter, FAST with Bounded
Rectification, PyCA culling + aggregation, orientation + descriptors, stereo
row matching) over one batch of synthetic input: the 100-frame KITTI-shaped
sequence (1241x376 u8, 8 levels, scale 1.2, FAST 20 with fallback 7, 32x32
cells, 2000 features per image) by default.

Modes: ``batched`` (all frames of the step in one launch sequence, the
headline) and ``plain`` (one C-ABI call per stereo pair).  Inputs are resident
in HBM before the timed region; L2 is flushed (256 MB write) before every
timed step.  ``e2e`` repeats the batched step through the C ABI with pinned
host images and downloads every result block, copies inside the timed region.

``--impl reference`` times the CPU oracle (the plain C implementation written
from the paper) on the host cores, one stereo pair per step.

Multi-GPU (torchrun): replicas only -- every rank processes its own copy of
the sequence with no data-path collective; value = pairs of all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stereo pairs/s (8-level FAST+BR+PyCA) plain vs batched vs learned-skip; % HBM peak"
UNIT = "stereo pairs/s"

WORKLOAD_DESC = {
    "kitti_1241x376_L8": "KITTI-shaped synthetic stereo sequence, 1241x376 u8, 8 levels at scale 1.2, "
                         "FAST 20 (fallback 7), 32x32 cells, 2000 features per image",
    "euroc_752x480_L8": "EuRoC-shaped synthetic stereo sequence, 752x480 u8, 8 levels at scale 1.2, "
                        "FAST 20 (fallback 7), 32x32 cells, 1200 features per image",
    "fhd_1920x1080_L8": "1920x1080 synthetic stereo sequence, 8 levels at scale 1.2, FAST 20 (fallback 7), "
                        "32x32 cells, 3000 features per image",
    "single_640x480_L1": "single 640x480 stereo pair, 1 level, FAST 20, 32x32 cells, 1 feature per cell",
}

# Stage -> kernel name, for the roofline and the ncu summaries.
KERNELS = {"pyramid": "k_pyramid", "detect": "k_fast_cull", "pfa_nms": "k_pfa_nms",
           "pfa_final": "k_pfa_finalize", "orb": "k_orient_desc", "match": "k_match"}
KERNEL_SOURCES = {"k_pyramid": "k_detect.cu", "k_fast_cull": "k_detect.cu", "k_pfa_nms": "k_pyca.cu",
                  "k_pfa_finalize": "k_pyca.cu", "k_orient_desc": "k_orb_match.cu", "k_match": "k_orb_match.cu"}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="kitti_1241x376_L8", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--frames", type=int, default=100)
    ap.add_argument("--mode", choices=["batched", "plain"], default="batched")
    ap.add_argument("--cpu-pairs", type=int, default=12, help="pairs in the oracle CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the batched mode only (no plain mode, no e2e): the launch sequence ncu captures")
    return ap.parse_args()


def workload_params(name):
    from paper_2410_04090_gb300 import scenes
    w = scenes.WORKLOADS[name]
    return dict(levels=w["levels"], scale=1.2, fast_thresh=w["fast_thresh"], cell=32, max_feats=w["max_feats"]), w


def make_frames(name, frames):
    from paper_2410_04090_gb300 import scenes
    return [scenes.workload_pair(name, f) for f in range(frames)]


# ------------------------------------------------------------------ helpers

def level_pixels(W0, H0, levels, scale):
    from paper_2410_04090_gb300 import jslam
    w, h, _ = jslam.level_geometry(W0, H0, levels, scale, 32)
    return [int(a) * int(b) for a, b in zip(w, h)]


def algorithmic_bytes(stage, W0, H0, jp, n_pairs, kp_counts):
    """Bytes a stage must move per launch (the batch's n_pairs pairs)."""
    px = level_pixels(W0, H0, jp["levels"], jp["scale"])
    A = sum(px)
    imgs = 2 * n_pairs
    kps = sum(kp_counts)
    if stage == "pyramid":   # read L0, write raw levels >= 1, write every blurred level
        return imgs * (px[0] + (A - px[0]) + A)
    if stage == "detect":    # read every raw level once
        return imgs * A
    if stage == "orb":       # per keypoint: 32-byte descriptor + angle + sector out
        return kps * (32 + 4 + 1)
    if stage == "match":     # per left keypoint: its descriptor and the result
        return (kps // 2) * (32 + 8)
    return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs"), "measured"
    except (OSError, ValueError):
        return 6800.0, "fallback"


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary of this kernel,
    or None if there is none or the kernel's source changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2410_04090_gb300", "csrc", KERNEL_SOURCES[kernel])
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if vals.get("source_sha256_16") != cur:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_workload"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------ reference arm

def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np
    from oracle import oracle as O
    jp, w = workload_params(args.workload)
    p = O.FrontendParams(levels=jp["levels"], max_feats=jp["max_feats"], fast_thresh=jp["fast_thresh"],
                         fast_thresh_lo=w["fast_thresh_lo"])
    frames = make_frames(args.workload, min(args.steps + args.warmup, args.frames))
    for i in range(args.warmup):
        fr = frames[i % len(frames)]
        O.extract_pair(fr.left, fr.right, p)
    times = []
    for i in range(args.steps):
        fr = frames[(args.warmup + i) % len(frames)]
        t0 = time.perf_counter()
        O.extract_pair(fr.left, fr.right, p)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_DESC[args.workload]}",
                       "step": "one stereo pair through the CPU oracle (bounded sample of the sequence)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} stereo pairs of the sequence, one per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def cpu_baseline(args, frames, jp, w):
    from oracle import oracle as O
    p = O.FrontendParams(levels=jp["levels"], max_feats=jp["max_feats"], fast_thresh=jp["fast_thresh"],
                         fast_thresh_lo=w["fast_thresh_lo"])
    n = min(args.cpu_pairs, len(frames))
    O.extract_pair(frames[0].left, frames[0].right, p)  # warm the library
    t0 = time.perf_counter()
    for i in range(n):
        O.extract_pair(frames[i].left, frames[i].right, p)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} stereo pairs of the sequence, single-threaded C oracle"}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    from paper_2410_04090_gb300 import build as B

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        if rank == 0:
            B.build()
        dist.barrier()
    else:
        torch.cuda.set_device(0)
        B.build()
    from paper_2410_04090_gb300 import jslam

    jp, w = workload_params(args.workload)
    frames = make_frames(args.workload, args.frames)
    W0, H0 = frames[0].left.shape[1], frames[0].left.shape[0]
    dev = torch.device("cuda", torch.cuda.current_device())
    lefts = [torch.from_numpy(f.left).to(dev) for f in frames]
    rights = [torch.from_numpy(f.right).to(dev) for f in frames]
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)  # torch work (flush, events) and the library share this stream
    fe = jslam.Frontend(device=dev.index, stream=stream, max_width=W0, max_height=H0, max_levels=8,
                        max_feats=jp["max_feats"], max_pairs=args.frames, fast_thresh_lo=w["fast_thresh_lo"])
    jobs = [jslam.Job(l, r, **jp) for l, r in zip(lefts, rights)]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2

    def step_batched():
        fe.extract_batch(jobs)
        fe.match()

    def step_plain():
        for l, r in zip(lefts, rights):
            fe.extract(l, r, **jp)
            fe.match()

    def timed(step, k, on_step=None):
        total = 0.0
        for i in range(k):
            flush.fill_(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            if on_step:
                on_step()
        return total  # ms

    modes = {"batched": step_batched, "plain": step_plain}
    if args.only_batched:
        args.mode = "batched"
        modes = {"batched": step_batched}
    main_step = modes[args.mode]
    for _ in range(args.warmup):
        for s in modes.values():
            s()
    torch.cuda.synchronize()

    # timed region: the headline mode, with per-stage events in batched mode
    fe.enable_stage_timing(args.mode == "batched")
    stage_acc = {k: 0.0 for k in jslam.STAGES}

    def grab():
        if args.mode == "batched":
            for k, v in fe.stage_times().items():
                stage_acc[k] += v

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clocks:
        total_ms = timed(main_step, args.steps, grab)
    fe.enable_stage_timing(False)
    other = "plain" if args.mode == "batched" else "batched"
    other_ms = timed(modes[other], args.steps) if other in modes else float("nan")

    t = torch.tensor([total_ms, other_ms], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms, other_ms = t.tolist()
    pairs = args.frames * args.steps * world
    value = pairs / (total_ms / 1e3)
    mode_values = {args.mode: value}
    if other in modes:
        mode_values[other] = pairs / (other_ms / 1e3)

    # keypoint counts of the last batch (for algorithmic bytes)
    fe.extract_batch(jobs); fe.match(); fe.sync()
    counts = [fe.keypoints(p, s)["count"] for p in range(args.frames) for s in (0, 1)]

    # end to end: pinned host images through the C ABI, result blocks back
    e2e_value, h2d, d2h = None, 0, 0
    if not args.only_batched:
        e2e_value, h2d, d2h = run_e2e(args, fe, frames, jp, jslam, torch, dist, dev, pairs)
    if rank == 0:
        emit(args, world, value, total_ms, mode_values, stage_acc, counts, W0, H0, jp, frames, w, e2e_value,
             h2d, d2h, clocks)
    fe.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_e2e(args, fe, frames, jp, jslam, torch, dist, dev, pairs):
    host_l = [torch.from_numpy(f.left).pin_memory() for f in frames]
    host_r = [torch.from_numpy(f.right).pin_memory() for f in frames]
    hjobs = [jslam.Job(l.numpy(), r.numpy(), **jp) for l, r in zip(host_l, host_r)]
    fe.extract_batch(hjobs); fe.match(); fe.sync()
    rb = [fe.result_bytes(p) for p in range(args.frames)]
    outs = [torch.empty(n, dtype=torch.uint8).pin_memory() for n in rb]

    def step_e2e():
        fe.extract_batch(hjobs)
        fe.match()
        for p in range(args.frames):
            fe.download(p, outs[p])
        fe.sync()

    for _ in range(args.warmup):
        step_e2e()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if dist:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = pairs / te.item()
    h2d = sum(f.left.nbytes + f.right.nbytes for f in frames)
    d2h = sum(rb)
    return e2e_value, h2d, d2h


def emit(args, world, value, total_ms, mode_values, stage_acc, counts, W0, H0, jp, frames, w, e2e_value, h2d,
     d2h, clocks):
    import numpy as np
    peak, peak_kind = measured_peaks()
    stage_ms = {k: v / args.steps for k, v in stage_acc.items()}
    roof = None
    if args.mode == "batched" and any(stage_ms.values()):
        dom = max((k for k in stage_ms if algorithmic_bytes(k, W0, H0, jp, 1, [1]) is not None),
                  key=lambda k: stage_ms[k])
        alg = algorithmic_bytes(dom, W0, H0, jp, args.frames, counts)
        ach = alg / (stage_ms[dom] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": KERNELS[dom], "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_kind": f"{peak_kind} HBM copy bandwidth",
                "algorithmic_bytes_per_launch": alg,
                "traffic": profiled_traffic(KERNELS[dom], args.workload),
                "stage_ms_per_launch": stage_ms}
    cpu = None if args.no_cpu_baseline else cpu_baseline(args, frames, jp, w)
    launches_per_call = 6
    gpu_launches = launches_per_call * args.steps * (1 if args.mode == "batched" else args.frames)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_DESC[args.workload]}",
                       "frames_per_step": args.frames, "mode": args.mode,
                       "parallelism": f"replicas x{world}", "l2": "flushed before every step (256 MB write)"},
            "modes": mode_values,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": None if e2e_value is None else
                   {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": clocks.summary(), "gpu_launches": gpu_launches,
            "keypoints_per_image_mean": float(np.mean(counts))}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
