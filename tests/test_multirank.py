"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): the barrier, the
max-over-ranks timer, the whole-job throughput of N replicas and the reference arm's
rank gating.  No GPU; the GPU path runs one replica per rank with the same helpers."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    t = 1.0 + rank                      # rank 1 is the slow one
    slowest = bench.max_over_ranks(t, world)
    rate = bench.job_throughput(100.0, t, world)
    bench.barrier(world)
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"slowest": slowest, "rate": rate}, f)
    dist.destroy_process_group()


def test_max_over_ranks_and_job_throughput(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        d = json.load(open(tmp_path / ("rank%d.json" % r)))
        assert d["slowest"] == 2.0
        assert d["rate"] == pytest.approx(100.0 * world / 2.0)


def test_reference_arm_prints_on_rank0_only(tmp_path):
    """Ranks other than 0 of `bench.py --impl reference` exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    """Rank 0 of `bench.py --impl reference` (world size 1) prints one JSON line with the
    contract's keys: the oracle timed on the host cores on a bounded sample, in the main
    arm's metric, unit and config, with an e2e entry that moves no bytes."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "views/s"
    assert d["config"]["workload"] == bench.WORKLOAD and d["higher_is_better"] is True
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 1, 0)
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
