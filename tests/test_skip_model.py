"""The committed learned-skip model has the layout jslam_set_skip_model
documents -- the 16-byte header {"JSKP", version 1, 16 channels, downsample
8}, FP32 biases b1[16], b2[16], b3[1], then BF16 weights of the 1 -> 16 -> 16
-> 1 stack of 3x3 convolutions -- with finite, non-trivial values, and its
training record meets the mode's recall bar on held-out frames."""
import json
import os
import struct

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2410_04090_gb300")


def test_blob_layout_and_values():
    blob = open(os.path.join(HERE, "skipnet_v1.bin"), "rb").read()
    magic, version, channels, down = struct.unpack("<4sIII", blob[:16])
    assert (magic, version, channels, down) == (b"JSKP", 1, 16, 8)
    n_w = 16 * 1 * 9 + 16 * 16 * 9 + 1 * 16 * 9
    assert len(blob) == 16 + 4 * (16 + 16 + 1) + 2 * n_w
    biases = np.frombuffer(blob, "<f4", 33, 16)
    bf16 = np.frombuffer(blob, "<u2", n_w, 16 + 4 * 33)
    weights = (bf16.astype(np.uint32) << 16).view(np.float32)
    assert np.isfinite(biases).all() and np.isfinite(weights).all()
    w1, w2, w3 = weights[:144], weights[144:144 + 2304], weights[144 + 2304:]
    for w in (w1, w2, w3):
        assert np.abs(w).max() > 1e-3 and np.abs(w).max() < 100.0


def test_training_record_meets_the_recall_bar():
    meta = json.load(open(os.path.join(HERE, "skipnet_v1.json")))
    assert np.isfinite(meta["thresh"])
    assert meta["levels"] == 8 and meta["cell"] == 32
    for kind in ("planes", "euroc"):
        assert meta["val"][kind]["occupied_cell_recall"] >= 0.99, kind
