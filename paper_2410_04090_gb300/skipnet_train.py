"""Train the learned cell-skip proposal and export its weight blob.

The net sees the 8x8 box mean of level 0 (scaled to [-0.5, 0.5]) and
predicts, per s0 culling cell, whether the exact path culls any corner (at
any level) whose s0 projection falls in the cell -- a cell without one can be
skipped without losing anything.  Labels come from the exact path itself
(libjslam with the proposal off, run without NMS suppression and without a
keypoint cap, so that its keypoints are exactly the per-cell culled corners)
on seeded synthetic frames of two kinds: the textured planes scenes (FHD) and
the EuRoC-shaped scenes with flat regions (752x480).  Held-out frames from
other scene seeds pick the logit threshold that keeps the requested fraction
of occupied cells.

Usage (needs a GPU for the labels):
    python -m paper_2410_04090_gb300.skipnet_train --frames 3000 --out skipnet_v1.bin

Writes the blob (header + FP32 biases + BF16 weights, the layout
jslam_set_skip_model reads) and a JSON sidecar with the threshold and the
training summary.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import struct
import sys
import time

import numpy as np

DOWN = 8
CHANNELS = 16


def box_mean(img: np.ndarray) -> np.ndarray:
    """8x8 block means (partial edge blocks average their valid pixels), scaled to [-0.5, 0.5]."""
    H, W = img.shape
    h8, w8 = (H + DOWN - 1) // DOWN, (W + DOWN - 1) // DOWN
    pad = np.zeros((h8 * DOWN, w8 * DOWN), np.float64)
    cnt = np.zeros_like(pad)
    pad[:H, :W] = img
    cnt[:H, :W] = 1.0
    s = pad.reshape(h8, DOWN, w8, DOWN).sum(axis=(1, 3))
    c = cnt.reshape(h8, DOWN, w8, DOWN).sum(axis=(1, 3))
    return (s / c / 255.0 - 0.5).astype(np.float32)


def _gen(args):
    kind, w, h, frame, stream, cfg = args
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2410_04090_gb300 import scenes
    pr = scenes.stereo_pair(kind, w, h, frame=frame, stream=stream, config_id=cfg)
    return pr.left, pr.right


def cell_labels(fe, jslam, torch, pairs, params, cell: int):
    """Per image: 1 where a culled corner of any level projects into the s0 cell."""
    out = []
    dev = torch.device("cuda", 0)
    B = 32
    for i in range(0, len(pairs), B):
        chunk = pairs[i:i + B]
        jobs = [jslam.Job(torch.from_numpy(l).to(dev), torch.from_numpy(r).to(dev), **params) for l, r in chunk]
        fe.extract_batch(jobs)
        fe.sync()
        for p in range(len(chunk)):
            for side in (0, 1):
                kp = fe.keypoints(p, side)
                X = kp["X"].cpu().numpy().astype(np.int64)
                Y = kp["Y"].cpu().numpy().astype(np.int64)
                H, W = chunk[p][side].shape
                lab = np.zeros(((H + cell - 1) // cell, (W + cell - 1) // cell), np.float32)
                lab[Y // cell, X // cell] = 1.0
                out.append(lab)
    return out


def build_model(torch):
    nn = torch.nn
    return nn.Sequential(nn.Conv2d(1, CHANNELS, 3, padding=1), nn.ReLU(),
                         nn.Conv2d(CHANNELS, CHANNELS, 3, padding=1), nn.ReLU(),
                         nn.Conv2d(CHANNELS, 1, 3, padding=1))


def forward_bf16(torch, model, x):
    """The net with the inference kernel's rounding points: the input and both
    activations rounded to BF16 (weights are BF16 already), wide accumulation."""
    def rnd(t):
        return t.to(torch.bfloat16).to(t.dtype)
    convs = [m for m in model if isinstance(m, torch.nn.Conv2d)]
    h = rnd(x)
    for i, c in enumerate(convs):
        h = torch.nn.functional.conv2d(h, c.weight.to(h.dtype), c.bias.to(h.dtype), padding=1)
        if i < len(convs) - 1:
            h = rnd(torch.relu(h))
    return h


def cell_logits(torch, model, x, cell: int, kernel_numerics: bool = False):
    """Largest 1/8-scale logit over each s0 cell (partial edge cells included)."""
    k = cell // DOWN
    y = forward_bf16(torch, model, x) if kernel_numerics else model(x)
    return torch.nn.functional.max_pool2d(y, k, stride=k, ceil_mode=True)


def export_blob(torch, model) -> bytes:
    convs = [m for m in model if isinstance(m, torch.nn.Conv2d)]
    head = b"JSKP" + struct.pack("<III", 1, CHANNELS, DOWN)
    biases = np.concatenate([c.bias.detach().float().cpu().numpy().ravel() for c in convs]).astype("<f4")
    weights = [c.weight.detach().to(torch.bfloat16).view(torch.int16).cpu().numpy().ravel().astype("<i2")
               for c in convs]
    return head + biases.tobytes() + b"".join(w.tobytes() for w in weights)


def round_weights_bf16(torch, model):
    with torch.no_grad():
        for m in model:
            if isinstance(m, torch.nn.Conv2d):
                m.weight.copy_(m.weight.to(torch.bfloat16).float())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", type=int, default=3000, help="training stereo pairs (split over the scene kinds)")
    ap.add_argument("--val", type=int, default=200, help="held-out stereo pairs (other scene seeds)")
    ap.add_argument("--levels", type=int, default=8)
    ap.add_argument("--cell", type=int, default=32)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--cell-recall", type=float, default=0.999, help="held-out occupied-cell recall to keep")
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--out", default="skipnet_v1.bin")
    args = ap.parse_args()

    t0 = time.time()
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2410_04090_gb300 import build, jslam
    build.build()
    kinds = [("planes", 1920, 1080), ("euroc", 752, 480)]
    big = 60000  # no keypoint cap: every culled corner is kept
    params = dict(levels=args.levels, scale=1.2, fast_thresh=20, cell=args.cell, max_feats=big)
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(args.workers)
    fe = jslam.Frontend(device=0, max_width=1920, max_height=1080, max_feats=big, max_pairs=32, fast_thresh_lo=7,
                        nms_q=1)

    def dataset(n, stream0):
        """Generate, label and reduce n pairs per kind in chunks (images are not kept)."""
        out = {}
        for kind, w, h in kinds:
            xs, ys = [], []
            for c0 in range(0, n, 256):
                jobs = [(kind, w, h, f % 25, stream0 + f // 25, 5) for f in range(c0, min(n, c0 + 256))]
                pairs = pool.map(_gen, jobs, chunksize=4)
                ys += cell_labels(fe, jslam, torch, pairs, params, args.cell)
                xs += [box_mean(img) for pr in pairs for img in pr]
            out[kind] = (xs, ys)
        return out

    train = dataset(args.frames // len(kinds), 0)
    val = dataset(args.val // len(kinds), 100000)
    t_gen = time.time() - t0
    pool.close()
    fe.close()
    dev = torch.device("cuda", 0)
    sets = [(torch.from_numpy(np.stack(train[k][0]))[:, None].to(dev),
             torch.from_numpy(np.stack(train[k][1]))[:, None].to(dev)) for k, _, _ in kinds]

    torch.manual_seed(0)
    model = build_model(torch).to(dev)
    opt = torch.optim.Adam(model.parameters(), lr=2e-3)
    pos = float(sum(float(Y.sum()) for _, Y in sets) / sum(Y.numel() for _, Y in sets))
    loss_fn = torch.nn.BCEWithLogitsLoss(pos_weight=torch.tensor([max(1.0, (1 - pos) / max(pos, 1e-6))], device=dev))
    for epoch in range(args.epochs):
        tot, cnt = 0.0, 0
        batches = []
        for si, (X, _) in enumerate(sets):
            perm = torch.randperm(X.shape[0], device=dev)
            batches += [(si, perm[i:i + 32]) for i in range(0, X.shape[0], 32)]
        order = torch.randperm(len(batches)).tolist()
        for bi in order:
            si, idx = batches[bi]
            X, Y = sets[si]
            opt.zero_grad()
            loss = loss_fn(cell_logits(torch, model, X[idx], args.cell), Y[idx])
            loss.backward()
            opt.step()
            tot += float(loss) * len(idx)
            cnt += len(idx)
        for g in opt.param_groups:
            g["lr"] *= 0.8
        print(f"epoch {epoch} loss {tot / cnt:.4f}", flush=True)

    # threshold on held-out frames, with the BF16-rounded weights the kernel uses
    round_weights_bf16(torch, model)
    occ, skipped = [], {}
    logits = {}
    with torch.no_grad():
        for k, _, _ in kinds:
            Xv = torch.from_numpy(np.stack(val[k][0]))[:, None].to(dev)
            Yv = torch.from_numpy(np.stack(val[k][1]))[:, None].to(dev)
            lv = cell_logits(torch, model, Xv, args.cell, kernel_numerics=True)
            logits[k] = (lv, Yv)
            occ.append(lv[Yv > 0.5].float().cpu().numpy())
    occ = np.concatenate(occ)
    thresh = float(np.quantile(occ, 1.0 - args.cell_recall)) if occ.size else 0.0
    for k, (lv, Yv) in logits.items():
        skipped[k] = {"cells_skipped": float((lv < thresh).float().mean()),
                      "empty_cells": float((Yv < 0.5).float().mean()),
                      "occupied_cell_recall": float((lv[Yv > 0.5] >= thresh).float().mean())}
    blob = export_blob(torch, model)
    with open(args.out, "wb") as f:
        f.write(blob)
    meta = {"thresh": thresh, "train_pairs": args.frames, "val_pairs": args.val,
            "kinds": [f"{k} {w}x{h}" for k, w, h in kinds], "levels": args.levels, "cell": args.cell,
            "label": "s0 cell holds a culled corner of any level (no NMS, no cap)",
            "val_cell_recall_target": args.cell_recall, "val": skipped,
            "occupied_fraction_train": pos, "seconds_generate": t_gen, "seconds_total": time.time() - t0}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
