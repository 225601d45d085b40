#!/usr/bin/env python3
"""Throughput of the stereo frontend hot path on GB300: stereo pairs/s.

One step = the whole hot path (pyramid + Gaussian filter, FAST with Bounded
Rectification, PyCA culling + aggregation, orientation + descriptors, stereo
row matching) over one batch of synthetic input: by default the 100-frame
KITTI-shaped sequence (1241x376 u8, 8 levels, scale 1.2, FAST 20 with
fallback 7, 32x32 cells, 2000 features per image).

Modes, each timed over the same steps:
  graph_streams8  the step's pairs split over eight contexts on eight
                  streams, each part captured once as a CUDA graph and
                  replayed (fork/join by events) -- the headline
  graph_streams4/2  the same with four and two parts
  streams8/4/2    the same parts as plain batched calls
  batched         all pairs of the step in one C-ABI call (one launch per stage)
  graph           the batched call captured once as a CUDA graph and replayed
  plain           one C-ABI call per stereo pair
  plain_graph     one C-ABI call per stereo pair, each a replay of a captured
                  single-pair graph pointed at that pair's frames
  learned_skip    batched, with the learned cell-skip proposal (approximate;
                  its feature recall against the exact path is reported)
Inputs are resident in HBM before the timed region; L2 is flushed (256 MB
write) before every timed step.  `e2e` repeats the step through the C ABI
with pinned host images and downloads every result block, copies inside
the timed region.

`roofline` is the dominant kernel's algorithmic bytes per launch over its
CUDA-event time against the measured HBM copy bandwidth; its `alu` entry
puts the same launch's executed instructions (from the committed ncu
summary of that kernel, when its source is unchanged) against the integer
issue rate of the SMs.  `cpu_baseline` is the CPU oracle on the host cores,
frame-parallel (one spawned process per core), with the single-threaded
figure beside it.

``--impl reference`` times the CPU oracle (the plain C implementation written
from the paper) frame-parallel on the host cores, one pair per core per step.

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
    "mixed16": "16 concurrent stereo streams: 4x 640x480 (4 levels), 4x 752x480 (5), 4x 1241x376 (6), "
               "4x 1920x1080 (8), scale 1.2, FAST 20 (fallback 7), 32x32 cells",
}

# Stage -> kernel name, for the roofline and the ncu summaries.
KERNELS = {"pyramid": "k_pyramid", "detect": "k_fast_bits", "pfa_nms": "k_pfa_nms",
           "pfa_final": "k_pfa_finalize", "orb": "k_orient_desc", "match": "k_match"}
KERNEL_SOURCES = {"k_pyramid": "k_detect.cu", "k_fast_cull": "k_detect.cu", "k_fast_bits": "k_detect.cu",
                  "k_pfa_nms": "k_pyca.cu",
                  "k_pfa_finalize": "k_pyca.cu", "k_orient_desc": "k_orb_match.cu", "k_match": "k_orb_match.cu",
                  "k_skipnet": "k_skipnet.cu"}
LAUNCHES_PER_CALL = 6  # pyramid, detect, PFA NMS, PFA final, ORB, match (exact path)
SKIP_MODEL = os.path.join(ROOT, "paper_2410_04090_gb300", "skipnet_v1.bin")
# the autotuner's cache of picks (keyed by GPU, configuration and batch shape)
TUNE_CACHE = os.environ.get("JSLAM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "jslam",
                                                              "tune.json"))
REFINE_BF = 386.1448  # fx * baseline (pixels x metres) of a KITTI-like stereo rig, for the depth output


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="kitti_1241x376_L8", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--frames", type=int, default=100, help="pairs per step (sequence workloads)")
    ap.add_argument("--mode", choices=["batched", "graph", "plain", "plain_graph", "streams2", "graph_streams2", "streams4",
                                       "graph_streams4", "streams8", "graph_streams8"],
                    default="graph_streams8", help="the headline mode (the others are timed beside it)")
    ap.add_argument("--cpu-pairs", type=int, default=12, help="pairs in the oracle CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", type=int, nargs=2, metavar=("W", "H"),
                    help="detection tile in pixels instead of the autotuner's pick (no autotune launches)")
    ap.add_argument("--only-batched", action="store_true",
                    help="time the batched mode only (no other modes, no e2e): the launch sequence ncu captures")
    return ap.parse_args()


def make_workload(name, frames):
    """(stereo pairs, per-pair parameters, fallback threshold) of one step."""
    from paper_2410_04090_gb300 import scenes
    if name == "mixed16":
        pairs, params = [], []
        for i, sp in enumerate(scenes.MIXED_STREAMS):
            pairs.append(scenes.stereo_pair(sp["kind"], sp["width"], sp["height"], frame=0, stream=i, config_id=4))
            params.append(dict(levels=sp["levels"], scale=1.2, fast_thresh=20, cell=32, max_feats=sp["max_feats"]))
        return pairs, params, 7
    w = scenes.WORKLOADS[name]
    pairs = [scenes.workload_pair(name, f % w["frames"]) for f in range(frames)]
    p = dict(levels=w["levels"], scale=1.2, fast_thresh=w["fast_thresh"], cell=32, max_feats=w["max_feats"])
    return pairs, [p] * len(pairs), w["fast_thresh_lo"]


# ------------------------------------------------------------------ helpers

def level_pixels(W0, H0, levels, scale):
    from paper_2410_04090_gb300 import jslam
    w, h, _ = jslam.level_geometry(W0, H0, levels, scale, 32)
    return [int(a) * int(b) for a, b in zip(w, h)]


def path_bytes_per_pair(pairs, params, counts):
    """Algorithmic bytes of the whole path per stereo pair, averaged over the
    batch: per image, level 0 read once, raw levels n >= 1 and blurred
    levels n >= 0 written once, 48 bytes per keypoint out (keypoint record +
    descriptor); `counts` holds the keypoints of image 2 p + side."""
    total = 0
    for i, (pr, p) in enumerate(zip(pairs, params)):
        px = level_pixels(pr.left.shape[1], pr.left.shape[0], p["levels"], p["scale"])
        A = sum(px)
        total += sum(px[0] + (A - px[0]) + A + 48 * counts[2 * i + s] for s in (0, 1))
    return total / max(len(pairs), 1)


ALG_OPS_DEFINITION = ("Eq. 1-3 per tested pixel, one pixel per lane: 16 ring differences, 32 labels (Eq. 1, "
                      "bright and dark), 32 bit inserts into the two 16-bit masks, 3 for the Eq. 3 table "
                      "look-ups (Sec. III) = 83; per corner 31 for the response (16 absolute values, 15 adds) "
                      "and 1 for the cell maximum (Sec. II-C-1)")


def alg_ops_per_pixel(corner_fraction):
    """Integer operations per tested pixel of the scalar formulation of FAST
    with Bounded Rectification and per-cell culling (see ALG_OPS_DEFINITION);
    loads are not counted."""
    return 16 + 32 + 32 + 3 + (31 + 1) * corner_fraction


def level_pixels_batch(pairs, params):
    """Pixels of every level of every image of the batch."""
    return sum(2 * sum(level_pixels(pr.left.shape[1], pr.left.shape[0], p["levels"], p["scale"]))
               for pr, p in zip(pairs, params))


def algorithmic_bytes(stage, pairs, params, kp_counts):
    """Bytes a stage must move per launch over the whole batch (None: not defined)."""
    if stage not in ("pyramid", "detect", "orb", "match"):
        return None
    kps = sum(kp_counts)
    if stage == "orb":     # per keypoint: 32-byte descriptor + angle + sector out
        return kps * (32 + 4 + 1)
    if stage == "match":   # per left keypoint: its descriptor and the result
        return (kps // 2) * (32 + 8)
    total = 0
    for pr, p in zip(pairs, params):
        px = level_pixels(pr.left.shape[1], pr.left.shape[0], p["levels"], p["scale"])
        A = sum(px)
        if stage == "pyramid":   # read L0, write raw levels >= 1, write every blurred level
            total += 2 * (px[0] + (A - px[0]) + A)
        else:                    # detect: read every raw level once
            total += 2 * A
    return total


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


def code_hash(path):
    """First 16 hex digits of the SHA-256 of a source file's code: comments
    and whitespace removed, so that only a change of the code makes an ncu
    summary taken from it stale."""
    import re
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()[:16]


def profile_summary(kernel, workload):
    """Key/value lines of the committed ncu summary of this kernel on this
    workload, or None if there is none or the kernel's source changed since."""
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
    return vals if vals.get("source_code_sha256_16") == code_hash(src) else None


def profile_number(vals, key):
    try:
        return float(vals[key].split()[0])
    except (TypeError, KeyError, ValueError, IndexError):
        return None


def alu_peak(dev_index):
    """Integer issue rate in lane-ops/s: SMs x 4 schedulers x 32 lanes x the
    maximum SM clock (measured file, else the GB300 maximum 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except (OSError, ValueError):
        pass
    return sms * 128 * mhz * 1e6, sms, mhz


def oracle_params(O, p, lo):
    return O.FrontendParams(levels=p["levels"], scale=p["scale"], max_feats=p["max_feats"],
                            fast_thresh=p["fast_thresh"], cell=p["cell"], fast_thresh_lo=lo)


# ------------------------------------------------------------------ reference arm

def max_over_ranks(dist, values, device):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    rank sets the whole-job time); identity without a process group."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_value(pairs_per_rank_step, steps, world, total_ms):
    """Stereo pairs/s of the whole job: every rank processes its own replica
    of the step's pairs, the time is the slowest rank's."""
    return pairs_per_rank_step * steps * world / (total_ms / 1e3)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_pair(job):
    """One stereo pair through the CPU oracle (pool worker)."""
    left, right, p, lo = job
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    O.extract_pair(left, right, oracle_params(O, p, lo))
    return 0


class OraclePool:
    """Frame-parallel oracle: one independent stereo pair per worker process
    (spawned, so that it is safe after CUDA initialisation)."""

    def __init__(self, cores):
        import multiprocessing as mp
        self.cores = cores
        self.pool = mp.get_context("spawn").Pool(cores)

    def run(self, pairs, params, lo):
        jobs = [(pr.left, pr.right, p, lo) for pr, p in zip(pairs, params)]
        t0 = time.perf_counter()
        self.pool.map(_oracle_pair, jobs, chunksize=1)
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, rank):
    """The oracle as it stands, frame-parallel on the host cores: each step
    is one bounded sample of the workload (one pair per core)."""
    if rank != 0:
        return
    cores = host_cores()
    pairs, params, lo = make_workload(args.workload, min(args.frames, cores))
    sample = [(pairs[i % len(pairs)], params[i % len(pairs)]) for i in range(cores)]
    pool = OraclePool(cores)
    for _ in range(args.warmup):
        pool.run([a for a, _ in sample], [b for _, b in sample], lo)
    total = 0.0
    for _ in range(args.steps):
        total += pool.run([a for a, _ in sample], [b for _, b in sample], lo)
    pool.close()
    value = args.steps * cores / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_DESC[args.workload]}",
                       "step": f"{cores} stereo pairs of the workload through the CPU oracle, one per core"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{cores} stereo pairs per step (the first {min(len(pairs), cores)} "
                                       f"pairs of the workload), one spawned process per core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def cpu_baseline(args, pairs, params, lo):
    """The oracle on the host cores: frame-parallel over all cores (the
    reported value) and single-threaded (kept beside it)."""
    from oracle import oracle as O
    n = min(args.cpu_pairs, len(pairs))
    O.extract_pair(pairs[0].left, pairs[0].right, oracle_params(O, params[0], lo))  # warm the library
    t0 = time.perf_counter()
    for i in range(n):
        O.extract_pair(pairs[i].left, pairs[i].right, oracle_params(O, params[i], lo))
    single = n / (time.perf_counter() - t0)
    cores = host_cores()
    m = min(len(pairs), 2 * cores)
    pool = OraclePool(cores)
    pool.run(pairs[:cores], params[:cores], lo)  # workers up and warm
    dt = pool.run(pairs[:m], params[:m], lo)
    pool.close()
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {m} stereo pairs of the workload, one spawned process per core",
            "single_core": {"value": single, "unit": UNIT, "cores": 1,
                            "sample": f"first {n} stereo pairs of the workload, one thread"}}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

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
    os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
    from paper_2410_04090_gb300 import jslam

    pairs, params, lo = make_workload(args.workload, args.frames)
    n = len(pairs)
    dev = torch.device("cuda", torch.cuda.current_device())
    lefts = [torch.from_numpy(f.left).to(dev) for f in pairs]
    rights = [torch.from_numpy(f.right).to(dev) for f in pairs]
    torch.cuda.synchronize()  # the uploads land before any context stream reads them
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)  # torch work (flush, events) and the library share this stream
    dims = dict(max_width=max(p.left.shape[1] for p in pairs), max_height=max(p.left.shape[0] for p in pairs),
                max_levels=8, max_feats=max(p["max_feats"] for p in params), max_pairs=n, fast_thresh_lo=lo)
    fe = jslam.Frontend(device=dev.index, stream=stream, **dims)
    jobs = fe.prepare_batch([jslam.Job(l, r, **p) for l, r, p in zip(lefts, rights, params)])
    if args.tile:
        fe.set_tuning(*args.tile)
        tuning = tuple(args.tile) + (0, 0, 0)
        tune_source = "--tile"
    else:
        tuning = fe.autotune(jobs, cache=TUNE_CACHE)
        tune_source = "cache hit" if fe.last_tune_hit else "tuned (stored in the cache)"
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2

    def step_batched():
        fe.extract_batch(jobs)
        fe.match()

    def step_plain():
        for l, r, p in zip(lefts, rights, params):
            fe.extract(l, r, **p)
            fe.match()

    graph_fe = None
    plain_graph_fe = None
    single_jobs = None

    def step_graph():
        graph_fe.graph_launch()

    def step_plain_graph():
        for j in single_jobs:
            plain_graph_fe.graph_launch(j)

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

    skip_fe = None

    def step_skip():
        skip_fe.extract_batch(jobs)
        skip_fe.match()

    modes = {"batched": step_batched}
    extra_fes = []
    if not args.only_batched and os.path.exists(SKIP_MODEL):
        skip_fe = jslam.Frontend(device=dev.index, stream=stream, **dims)
        skip_fe.set_tuning(*tuning)
        skip_fe.set_skip_model(open(SKIP_MODEL, "rb").read(),
                               json.load(open(os.path.splitext(SKIP_MODEL)[0] + ".json"))["thresh"])
        modes["learned_skip"] = step_skip
    if not args.only_batched:
        graph_fe = jslam.Frontend(device=dev.index, stream=stream, **dims)
        graph_fe.set_tuning(*tuning)
        graph_fe.graph_capture(jobs)
        modes["graph"] = step_graph
        modes["plain"] = step_plain
        if len({(p.left.shape, tuple(sorted(q.items()))) for p, q in zip(pairs, params)}) == 1:
            # one stereo pair per call, each call one replay of a single-pair
            # graph pointed at that pair's frames
            plain_graph_fe = jslam.Frontend(device=dev.index, stream=stream, **dict(dims, max_pairs=1))
            plain_graph_fe.set_tuning(*tuning)
            single_jobs = [plain_graph_fe.prepare_batch([jslam.Job(l, r, **p)])
                           for l, r, p in zip(lefts, rights, params)]
            plain_graph_fe.graph_capture(single_jobs[0])
            modes["plain_graph"] = step_plain_graph
    def split_modes(S):
        """The step's pairs split over S contexts on S streams (fork and join
        on the timing stream): one part's kernels fill the others' launch
        gaps and kernel tails.  Returns (plain step, graph-replay step)."""
        bounds = [round(i * n / S) for i in range(S + 1)]
        streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(S - 1)]
        plain, graphs, parts = [], [], []
        for i in range(S):
            sl = slice(bounds[i], bounds[i + 1])
            d = dict(dims, max_pairs=max(1, bounds[i + 1] - bounds[i]))
            fp = jslam.Frontend(device=dev.index, stream=streams[i], **d)
            fg = jslam.Frontend(device=dev.index, stream=streams[i], **d)
            part = fp.prepare_batch([jslam.Job(l, r, **p) for l, r, p in zip(lefts[sl], rights[sl], params[sl])])
            for c in (fp, fg):
                c.set_tuning(*tuning)
            fg.graph_capture(part)
            plain.append(fp); graphs.append(fg); parts.append(part)
            extra_fes.extend([fp, fg])

        def fork_join(body):
            ev = torch.cuda.Event()
            ev.record(stream)
            for s_ in streams[1:]:
                s_.wait_event(ev)
            body()
            for s_ in streams[1:]:
                e_ = torch.cuda.Event()
                e_.record(s_)
                stream.wait_event(e_)

        def step_plain_split():
            def body():
                for fp, part in zip(plain, parts):
                    fp.extract_batch(part)
                    fp.match()
            fork_join(body)

        def step_graph_split():
            fork_join(lambda: [fg.graph_launch() for fg in graphs])

        return step_plain_split, step_graph_split

    if not args.only_batched:
        for S in (2, 4, 8):
            if n >= S:
                modes[f"streams{S}"], modes[f"graph_streams{S}"] = split_modes(S)
    if args.mode not in modes:
        args.mode = "batched"
    for _ in range(args.warmup):
        for s in modes.values():
            s()
    torch.cuda.synchronize()

    # timed regions: the headline mode first, then every other mode; the
    # batched mode's steps carry per-stage events (the per-kernel durations
    # of the roofline)
    stage_acc = {k: 0.0 for k in jslam.STAGES}

    def grab():
        for k, v in fe.stage_times().items():
            stage_acc[k] += v

    def timed_mode(m):
        fe.enable_stage_timing(m == "batched")
        ms = timed(modes[m], args.steps, grab if m == "batched" else None)
        fe.enable_stage_timing(False)
        return ms

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clocks:  # samples every timed region (all modes)
        time.sleep(0.3)  # let the sampler start before the first timed step
        total_ms = timed_mode(args.mode)
        other_ms = {m: timed_mode(m) for m in modes if m != args.mode}

    vals = max_over_ranks(dist, [total_ms] + list(other_ms.values()), dev)
    total_ms = vals[0]
    pairs_done = n * args.steps * world
    value = whole_job_value(n, args.steps, world, total_ms)
    mode_values = {args.mode: value}
    for m, ms in zip(other_ms, vals[1:]):
        mode_values[m] = whole_job_value(n, args.steps, world, ms)

    # keypoint counts of the last batch (for algorithmic bytes)
    fe.extract_batch(jobs); fe.match(); fe.sync()
    counts = [fe.keypoints(p, s)["count"] for p in range(n) for s in (0, 1)]
    skip_quality = None
    if skip_fe:
        skip_fe.extract_batch(jobs); skip_fe.sync()
        inter = total = kept = 0
        skipped = []
        for p in range(n):
            skipped.append(float(skip_fe.skip_view(p, 0)["skip"].float().mean()))
            for s in (0, 1):
                a = jslam.to_numpy(fe.keypoints(p, s)); b = jslam.to_numpy(skip_fe.keypoints(p, s))
                ka = set(zip(a["level"].tolist(), a["y"].tolist(), a["x"].tolist()))
                kb = set(zip(b["level"].tolist(), b["y"].tolist(), b["x"].tolist()))
                inter += len(ka & kb); total += len(ka); kept += len(kb)
        skip_quality = {"recall": inter / max(total, 1), "precision": inter / max(kept, 1),
                        "cells_skipped": sum(skipped) / len(skipped), "model": os.path.basename(SKIP_MODEL)}
        # the skip net's tensor-core work: 3x3 convs 1->16->16->1 per 1/8-scale position
        skip_fe.enable_stage_timing(True)
        skip_ms = []
        for _ in range(3):
            skip_fe.extract_batch(jobs); skip_fe.sync()
            skip_ms.append(skip_fe.stage_times()["skip"])
        skip_fe.enable_stage_timing(False)
        flop = sum(2 * ((pr.left.shape[0] + 7) // 8) * ((pr.left.shape[1] + 7) // 8) * 2 * (9 * 16 + 144 * 16 + 144)
                   for pr in pairs)
        ms = statistics.median(skip_ms)
        bf16_peak = None
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                bf16_peak = json.load(f).get("bf16_tflops")
        except (OSError, ValueError):
            pass
        tflops = flop / (ms / 1e3) / 1e12 if ms > 0 else None
        skip_quality["skipnet"] = {"kernel": "k_skipnet (tcgen05.mma kind::f16, BF16 in, FP32 accumulate)",
                                   "stage_ms": ms, "flop_per_launch": flop, "achieved_tflops": tflops,
                                   "peak_tflops": bf16_peak,
                                   "frac": (tflops / bf16_peak) if (tflops and bf16_peak) else None,
                                   "peak_kind": "measured cuBLAS bf16 burst"}

    # correlation minimisation (the middle-end's sub-pixel refinement, a step
    # beyond the hot path): timed beside the headline on the batched context
    refine = None
    if not args.only_batched:
        ref_ms = []

        def step_refine():
            fe.extract_batch(jobs)
            fe.match()
            fe.refine_matches(5, 5, REFINE_BF)

        fe.enable_stage_timing(True)
        ref_total = timed(step_refine, args.steps, lambda: ref_ms.append(fe.stage_times()["refine"]))
        fe.enable_stage_timing(False)
        fe.sync()
        matched = sum(int((fe.matches(p)["right_idx"] >= 0).sum()) for p in range(n))
        kept = sum(int((fe.refined(p)["disparity"] >= 0).sum()) for p in range(n))
        refine = {"stage_ms": statistics.median(ref_ms), "value_with_refine": n * args.steps / (ref_total / 1e3),
                  "unit": UNIT, "mode": "batched + jslam_refine_matches(half_window 5, search 5)",
                  "refined_fraction_of_matches": kept / max(matched, 1)}

    # feature tracking by projection (middle-end): frame k's left keypoints,
    # predicted at their own s0 positions, tracked into frame k + 1's left image
    track = None
    if not args.only_batched and n >= 2:
        fe.extract_batch(jobs); fe.sync()
        qs = []
        import numpy as np
        for k in range(n - 1):
            kp = jslam.to_numpy(fe.keypoints(k, 0))
            c = kp["count"]
            up = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a[:c], dt)).to(dev)
            qs.append((up(kp["X"], np.float32), up(kp["Y"], np.float32), up(kp["level"], np.uint8),
                       up(np.asarray(kp["desc"], np.uint32).view(np.int32), np.int32)))
        n_q = sum(int(q[0].numel()) for q in qs)
        hits = []

        def step_track():
            hits.clear()
            for k, (u, v, lv, dsc) in enumerate(qs):
                hits.append(fe.track(k + 1, 0, u, v, lv, dsc, 8.0, 100)[0])

        for _ in range(2):
            step_track()
        track_ms = timed(step_track, min(args.steps, 10))
        fe.sync()
        tracked = sum(int((h >= 0).sum()) for h in hits)
        track = {"queries_per_step": n_q, "calls_per_step": n - 1, "ms_per_step": track_ms / min(args.steps, 10),
                 "queries_per_s": n_q / (track_ms / min(args.steps, 10) / 1e3), "tracked_fraction": tracked / max(n_q, 1),
                 "mode": "jslam_track(radius 8, max_dist 100), previous frame's left keypoints into the next frame"}

    # the paper's feature-culling kernels (CRF-matrix + MLPT/TEWA) as an
    # ablation beside the fused detection kernel, on the same batch
    fc_abl = None
    if not args.only_batched:
        crf, fc = [], []
        fe.extract_batch(jobs)
        for _ in range(5):
            fe.fc_ablation(8)
            fe.sync()
            t = fe.fc_ablation_times()
            crf.append(t["crf_ms"]); fc.append(t["fc_ms"])
        # corner fraction of the first pair (primary threshold, every level), for the algorithmic op count
        corners = px = 0
        for side in (0, 1):
            for lv in range(params[0]["levels"]):
                c = fe.crf(0, side, lv).cpu().numpy()  # (torch has no uint16 compare on the GPU)
                corners += int((c > 0).sum())
                px += c.size
        fc_abl = {"crf_matrix_ms": statistics.median(crf[1:]), "mlpt_tewa_fc_ms": statistics.median(fc[1:]),
                  "corner_fraction_pair0": corners / max(px, 1),
                  "n_max": 8, "fused_detect_ms": stage_acc["detect"] / args.steps,
                  "note": "paper scheme: CRF-matrix of every level written to HBM (primary threshold), then "
                          "per-level MLPT/TEWA culling kernels; fused: FAST + BR + culling + PFA scatter in one "
                          "persistent kernel, no CRF-matrix"}

    # repeatability of Bounded Rectification against plain FAST on rotated
    # labeled scenes (the corner sets from the library's CRF-matrix)
    br_rep = None
    if not args.only_batched and rank == 0:
        from paper_2410_04090_gb300 import repeatability
        r = repeatability.study(device=dev.index)
        br_rep = {"angles_deg": r["angles"], "match_radius_px": r["radius_px"], "size": r["size"],
                  "eps": r["eps"], "labeled_corners_per_scene": r["corners_per_scene"],
                  "crf_ms_per_batch_of_angles": r["crf_ms"]}
        for set_name in repeatability.SCENES:
            br_rep[set_name] = {name: {"p_max": d["p_max"], "mean_f1": d["mean_f1"],
                                       "f1": [round(v, 4) for v in d["f1"]]}
                                for name, d in r[set_name].items()}

    e2e = None
    if not args.only_batched:
        e2e = run_e2e(args, pairs, params, jslam, torch, dist, dev, pairs_done, dims, tuning)
    if rank == 0:
        emit(args, world, n, value, total_ms, mode_values, stage_acc, counts, pairs, params, lo, e2e, clocks,
             tuning, skip_quality, dev.index, refine, track, fc_abl, br_rep, tune_source)
    fe.close()
    for extra in [graph_fe, skip_fe, plain_graph_fe] + extra_fes:
        if extra:
            extra.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


E2E_ROUTES = (("graph_parts4", 4, True), ("graph_parts8", 8, True), ("graph", 1, True), ("extract", 1, False))


def run_e2e(args, pairs, params, jslam, torch, dist, dev, pairs_done, dims, tuning):
    """End to end through the C ABI: every step uploads that step's frames
    from pinned host memory (one buffer holding all frames back to back, so
    the library moves each part's frames with one copy), extracts, matches
    and downloads the result blocks (one ranged copy per part), timed by the
    wall clock.  Routes: `extract` calls jslam_extract_batch + jslam_match
    per step; `graph` replays a graph captured on the host frames (the
    upload copy is a node of the graph, so every replay copies the frames
    again); `graph_parts4` and `graph_parts8` split the step's pairs over
    four and eight such graphs on their own streams.  Each route has two sets of contexts that take alternate
    steps, so one step's copies overlap the other's kernels; the headline
    is the first route, the others and a single-context figure (the
    extract route, one set, no overlap) ride along."""
    n = len(pairs)
    sizes = [(f.left.shape, f.right.shape) for f in pairs]
    total = sum(a[0] * a[1] + b[0] * b[1] for a, b in sizes)
    flat = torch.empty(total, dtype=torch.uint8).pin_memory()
    flat_np = flat.numpy()
    views, off = [], 0
    for f in pairs:
        pv = []
        for img in (f.left, f.right):
            v = flat_np[off: off + img.size].reshape(img.shape)
            v[...] = img
            pv.append(v)
            off += img.size
        views.append(pv)

    def make_route(parts, use_graph, sets=2):
        bounds = [round(i * n / parts) for i in range(parts + 1)]
        groups = []
        for _ in range(sets):
            g = []
            for i in range(parts):
                sl = slice(bounds[i], bounds[i + 1])
                if sl.start == sl.stop:
                    continue
                c = jslam.Frontend(device=dev.index, stream=torch.cuda.Stream(device=dev),
                                   **dict(dims, max_pairs=sl.stop - sl.start))
                c.set_tuning(*tuning)
                hj = c.prepare_batch([jslam.Job(v[0], v[1], **p) for v, p in zip(views[sl], params[sl])])
                if use_graph:
                    c.graph_capture(hj)
                else:
                    c.extract_batch(hj); c.match()
                c.sync()
                nb, _ = c.result_range(0, sl.stop - sl.start)
                g.append((c, hj, sl.stop - sl.start, torch.empty(nb, dtype=torch.uint8).pin_memory()))
            groups.append(g)

        def step(k):
            for c, hj, m, out in groups[k % len(groups)]:
                if use_graph:
                    c.graph_launch()
                else:
                    c.extract_batch(hj); c.match()
                c.download_range(0, m, out)

        def run(steps):
            for i in range(steps):
                step(i)
            for g in groups:
                for c, _, _, _ in g:
                    c.sync()
        return run, sum(out.numel() for _, _, _, out in groups[0]), [c for g in groups for c, _, _, _ in g]

    def timed(route):
        run, d2h, ctxs = route
        d2h_bytes.append(d2h)
        run(args.warmup)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        run(args.steps)
        dt = time.perf_counter() - t0
        for c in ctxs:  # one route's contexts at a time on the device
            c.close()
        return dt

    d2h_bytes = []
    secs = {name: timed(make_route(parts, use_graph)) for name, parts, use_graph in E2E_ROUTES}
    secs["single_context"] = timed(make_route(1, False, sets=1))
    names = list(secs)
    secs = dict(zip(names, max_over_ranks(dist, [secs[k] for k in names], dev)))
    head = E2E_ROUTES[0][0]
    res = {"value": pairs_done / secs[head], "unit": UNIT, "h2d_bytes_per_step": total,
           "d2h_bytes_per_step": d2h_bytes[0],
           "how": f"C ABI, pinned host frames, route {head}: the step's pairs in four parts, each part one replay "
                  "of a graph captured on its host frames (one upload copy inside the graph) on its own stream, "
                  "then one ranged result download per part; two sets of contexts take alternate steps; "
                  "wall clock",
           "routes": {k: pairs_done / v for k, v in secs.items()}}
    return res


def emit(args, world, n, value, total_ms, mode_values, stage_acc, counts, pairs, params, lo, e2e, clocks, tuning,
         skip_quality, dev_index, refine=None, track=None, fc_abl=None, br_rep=None, tune_source="--tile"):
    import numpy as np
    peak, peak_kind = measured_peaks()
    stage_ms = {k: v / args.steps for k, v in stage_acc.items()}
    roof = None
    if any(stage_ms.values()):
        dom = max((k for k in stage_ms if algorithmic_bytes(k, pairs[:1], params[:1], [1]) is not None),
                  key=lambda k: stage_ms[k])
        alg = algorithmic_bytes(dom, pairs, params, counts)
        ach = alg / (stage_ms[dom] / 1e3) / 1e9
        prof = profile_summary(KERNELS[dom], args.workload)
        hbm = {"bound": "hbm", "kernel": KERNELS[dom], "achieved": ach, "peak": peak, "unit": "GB/s",
               "frac": ach / peak, "peak_kind": f"{peak_kind} HBM copy bandwidth",
               "algorithmic_bytes_per_launch": alg,
               "traffic": profile_number(prof, "dram_bytes_per_launch_full_workload")}
        roof = hbm
        # the kernels of the path are integer-issue bound: with the launch's
        # executed instructions from the committed ncu summary, the roofline
        # is the issue rate, and the HBM view rides along
        warp_inst = profile_number(prof, "inst_executed_warp_per_launch")
        if warp_inst:
            apeak, sms, mhz = alu_peak(dev_index)
            lane_ops = warp_inst * 32
            pixels = level_pixels_batch(pairs, params)
            rate = lane_ops / (stage_ms[dom] / 1e3)
            roof = {"bound": "alu", "kernel": KERNELS[dom], "achieved": rate, "peak": apeak, "unit": "lane-op/s",
                    "frac": rate / apeak, "peak_kind": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz (integer issue)",
                    "traffic": hbm["traffic"], "inst_per_launch": lane_ops, "ops_per_pixel": lane_ops / pixels,
                    "instructions_from": f"profiles/{KERNELS[dom]}_{args.workload}.txt",
                    "hbm": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "peak_kind",
                                                "algorithmic_bytes_per_launch")}}
        roof["stage_ms_per_launch"] = stage_ms
        roof["stage_timing"] = "CUDA events on the context stream between the stages of the batched mode's timed steps"
    per_pair = path_bytes_per_pair(pairs, params, counts)
    path_hbm = {"algorithmic_bytes_per_pair": per_pair, "achieved": per_pair * value / 1e9, "peak": peak,
                "unit": "GB/s", "frac": per_pair * value / 1e9 / peak,
                "definition": "A0 (1 + (S_L - 1) + S_L) + 48 N_kp per image, at the headline pairs/s",
                "by_mode": {m: {"pairs_per_s": v, "achieved": per_pair * v / 1e9, "frac": per_pair * v / 1e9 / peak}
                            for m, v in mode_values.items()}}
    if roof and roof.get("bound") == "alu" and fc_abl and "corner_fraction_pair0" in fc_abl:
        f = fc_abl["corner_fraction_pair0"]
        alg = alg_ops_per_pixel(f)
        pixels = level_pixels_batch(pairs, params)
        rate = alg * pixels / (stage_ms["detect"] / 1e3)
        roof["algorithmic"] = {"ops_per_pixel": alg, "corner_fraction": f, "achieved": rate, "frac": rate / roof["peak"],
                               "definition": ALG_OPS_DEFINITION}
    cpu = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(args, pairs, params, lo)
    launches = {"batched": LAUNCHES_PER_CALL, "graph": LAUNCHES_PER_CALL, "plain": LAUNCHES_PER_CALL * n,
                "plain_graph": LAUNCHES_PER_CALL * n,
                "learned_skip": LAUNCHES_PER_CALL + 2, "streams2": 2 * LAUNCHES_PER_CALL,
                "graph_streams2": 2 * LAUNCHES_PER_CALL, "streams4": 4 * LAUNCHES_PER_CALL,
                "graph_streams4": 4 * LAUNCHES_PER_CALL, "streams8": 8 * LAUNCHES_PER_CALL,
                "graph_streams8": 8 * LAUNCHES_PER_CALL}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {WORKLOAD_DESC[args.workload]}",
                       "pairs_per_step": n, "mode": args.mode, "detect_tile_px": list(tuning[:2]),
                       "tuning": {"nms_kernel": tuning[2], "detect_ctas_per_sm": tuning[3],
                                  "tile_order": tuning[4],
                                  "source": tune_source},
                       "parallelism": f"replicas x{world}", "l2": "flushed before every step (256 MB write)"},
            "modes": mode_values, "learned_skip": skip_quality, "refine": refine, "track": track,
            "fc_ablation": fc_abl, "br_repeatability": br_rep,
            "roofline": roof, "path_hbm": path_hbm, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clocks.summary(), "gpu_launches": launches[args.mode] * args.steps,
            "keypoints_per_image_mean": float(np.mean(counts))}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
