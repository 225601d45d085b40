"""The committed ncu summaries stay reproducible and usable: each names its
kernel and workload, gives a command that keeps the clocks unlocked and runs
only committed files with arguments bench.py still accepts, carries the
figures the benchmark reads and the hash of the source it was taken from."""
import os
import shlex
import sys
from unittest import mock

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SUMMARIES = sorted(f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".txt"))


def _fields(name):
    vals = {}
    for ln in open(os.path.join(ROOT, "profiles", name)).read().splitlines():
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    return vals


@pytest.mark.parametrize("name", SUMMARIES)
def test_summary_is_reproducible_and_current(name):
    v = _fields(name)
    assert name == f"{v['kernel']}_{v['workload']}.txt"
    for key in ("gpu_time_ms", "dram_bytes_per_launch_full_workload", "inst_executed_warp_per_launch",
                "registers_per_thread"):
        assert bench.profile_number(v, key) is not None, key
    cmd = shlex.split(v["command"])
    assert cmd[0] == "ncu" and "--clock-control" in cmd and cmd[cmd.index("--clock-control") + 1] == "none"
    i = cmd.index("bench.py")
    assert cmd[i - 1] == "python" and os.path.exists(os.path.join(ROOT, "bench.py"))
    with mock.patch.object(sys, "argv", ["bench.py"] + cmd[i + 1:]):
        args = bench.parse_args()
    assert args.workload == v["workload"]
    # the hash of the kernel's source at capture time; a summary whose kernel changed since is
    # ignored by the benchmark (it falls back to the HBM view), so staleness is allowed here
    h = v["source_code_sha256_16"]
    assert len(h) == 16 and all(ch in "0123456789abcdef" for ch in h)
    assert v["source_file"] == "paper_2410_04090_gb300/csrc/" + bench.KERNEL_SOURCES[v["kernel"]]


def test_launch_list_command_keeps_clocks_unlocked():
    text = open(os.path.join(ROOT, "profiles", "launches_kitti_1241x376_L8_batched.md")).read()
    assert "--clock-control none" in text and "python bench.py" in text
