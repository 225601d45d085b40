"""Repeatability of Bounded Rectification on rotated labeled scenes.

The paper measures corner quality on synthetic images with known corners,
rotated through the full circle, as the F1 score of the detected corners,
Bounded Rectification against plain FAST (Sec. IV-A and its repeatability
figure).  This module runs that study on the library:

* scenes: ``scenes.corner_scene`` -- convex polygons with labeled vertices,
  rotated by each angle about the image centre; a second set adds unlabeled
  1-2 px dots, the specks of real images that are not corners;
* corners: the CRF-matrix of a one-level extraction (Eq. 1-3 at the primary
  threshold, every pixel, before culling), read with ``jslam_crf_view`` after
  ``jslam_fc_ablation``; (P_min, P_max) = (9, 13) is Bounded Rectification,
  (9, 16) the unbounded FAST of Eq. 2;
* score: a corner pixel is a detection at its centre; a detection is correct
  when a labeled vertex lies within ``RADIUS`` px, a vertex is found when a
  detection lies within ``RADIUS`` px; precision and recall are over the two
  sets (no one-to-one assignment) and F1 is their harmonic mean.
"""
from __future__ import annotations

import numpy as np

from . import scenes

ANGLES = tuple(range(-175, 176, 25))  # the paper's rotation axis: -175 .. 175 degrees in steps of 25
RADIUS = 3.0
SIZE = (480, 360)
SEED = 2410
P_MAX = {"bounded_rectification": 13, "plain_fast": 16}
SCENES = {"polygons": 0, "polygons_and_dots": 40}  # scene set -> unlabeled dots per image


def detections(crf) -> np.ndarray:
    """Centres (x + 0.5, y + 0.5) of the pixels with a non-zero response."""
    ys, xs = np.nonzero(np.asarray(crf))
    return np.stack([xs + 0.5, ys + 0.5], axis=1).astype(np.float64)


def f1(det: np.ndarray, gt: np.ndarray, radius: float = RADIUS):
    """(precision, recall, F1) of detections `det` [N, 2] against labeled
    corners `gt` [M, 2]; 0 where a set is empty."""
    det = np.asarray(det, np.float64).reshape(-1, 2)
    gt = np.asarray(gt, np.float64).reshape(-1, 2)
    if len(det) == 0 or len(gt) == 0:
        return 0.0, 0.0, 0.0
    d2 = ((det[:, None, :] - gt[None, :, :]) ** 2).sum(axis=2)
    near = d2 <= radius * radius
    precision = float(near.any(axis=1).mean())
    recall = float(near.any(axis=0).mean())
    score = 0.0 if precision + recall == 0 else 2 * precision * recall / (precision + recall)
    return precision, recall, score


def study(angles=ANGLES, eps: int = 20, seed: int = SEED, size=SIZE, device: int = 0, border: int = 19):
    """F1 per angle of both detectors on both scene sets, on the GPU, and the
    CRF kernel's time.

    Returns {scene set: {detector: {"p_max", "f1": [...], "precision":
    [...], "recall": [...], "mean_f1"}}, "angles": [...],
    "corners_per_scene": n, "crf_ms": ms per batch of len(angles) images}."""
    import torch

    from . import jslam

    W, H = size
    dev = torch.device("cuda", device)
    out = {"angles": list(angles), "radius_px": RADIUS, "size": [W, H], "eps": eps}
    crf_ms = []
    for set_name, dots in SCENES.items():
        sc = [scenes.corner_scene(W, H, a, seed, dots=dots) for a in angles]
        imgs = [torch.from_numpy(s.image).to(dev) for s in sc]
        out["corners_per_scene"] = int(len(sc[0].corners))
        res = {}
        for name, p_max in P_MAX.items():
            fe = jslam.Frontend(device=device, max_width=W, max_height=H, max_feats=4000, max_pairs=len(angles),
                                p_min=9, p_max=p_max, border=border, fast_thresh_lo=0)
            try:
                jobs = fe.prepare_batch([jslam.Job(im, im, levels=1, scale=1.2, fast_thresh=eps, cell=32,
                                                   max_feats=4000) for im in imgs])
                fe.extract_batch(jobs)
                fe.fc_ablation(8)
                fe.sync()
                crf_ms.append(fe.fc_ablation_times()["crf_ms"])
                rows = [f1(detections(fe.crf(i, 0, 0).cpu().numpy()), s.corners) for i, s in enumerate(sc)]
            finally:
                fe.close()
            res[name] = {"p_max": p_max, "precision": [r[0] for r in rows], "recall": [r[1] for r in rows],
                         "f1": [r[2] for r in rows], "mean_f1": float(np.mean([r[2] for r in rows]))}
        out[set_name] = res
    out["crf_ms"] = float(np.mean(crf_ms))
    return out
