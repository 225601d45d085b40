"""The multi-rank parts of bench.py, on CPU: replicas only (no data-path
collective), the slowest rank's time for the whole job, rank 0 alone prints
and runs the reference arm.  Two gloo ranks on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (10 + r) ms for the headline and (30 - r) ms for another mode
    vals = bench.max_over_ranks(dist, [10.0 + rank, 30.0 - rank], "cpu")
    q.put((rank, vals, bench.whole_job_value(100, 5, world, vals[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get() for _ in range(2))
    for rank, vals, value in got:
        assert vals == [11.0, 30.0]                 # the slowest rank of each mode
        assert value == pytest.approx(100 * 5 * 2 / 0.011)  # all ranks' pairs over that time
    assert bench_single() == pytest.approx(100 * 5 / 0.010)


def bench_single():
    sys.path.insert(0, ROOT)
    import bench
    (v,) = bench.max_over_ranks(None, [10.0], "cpu")
    return bench.whole_job_value(100, 5, 1, v)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--workload", "single_640x480_L1"]
    r1 = subprocess.run(cmd, env=dict(env, RANK="1", LOCAL_RANK="1"), capture_output=True, text=True, timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(cmd, env=dict(env, RANK="0", LOCAL_RANK="0"), capture_output=True, text=True, timeout=300)
    assert r0.returncode == 0
    lines = [l for l in r0.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["value"] > 0
    # the rest of the line's contract: the same metric, unit and direction as our arm
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT == d["e2e"]["unit"]
    assert (d["steps"], d["warmup"], d["higher_is_better"], d["scaling"]) == (1, 0, True, "weak")
    assert d["vs_baseline"] is None and d["data"] == "synthetic" and d["ms_per_step"] > 0
    assert d["config"]["workload"].startswith("single_640x480_L1")
    cb = d["cpu_baseline"]
    assert cb["value"] == d["value"] == d["e2e"]["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"]["d2h_bytes_per_step"] == 0
