"""Host logic of the multi-process benchmark path, as two gloo ranks on the CPU.

The path shards into independent replicas (one field per rank, no data
exchange), so what the ranks share is host logic only: every rank reports the
slowest rank's time, the whole-job throughput counts the bytes of all ranks,
and the reference arm runs on rank 0 alone while the other ranks exit at once.
"""
import json
import os
import socket
import subprocess
import sys
import tempfile

import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [12.5, 30.0, 7.0, 18.0][rank]
    ms = bench.max_over_ranks(local_ms, "cpu")
    gbs = bench.job_gbs(world, 2.0e9, ms)
    dist.barrier()
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"ms": ms, "gbs": gbs}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_job_throughput():
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True,
                           start_method="spawn")
        res = [json.load(open(os.path.join(d, "r%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["ms"] == 30.0
        # two ranks x 2 GB per step in 30 ms
        assert abs(r["gbs"] - 2 * 2.0e9 / 0.030 / 1e9) < 1e-9


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(4.25, "cpu") == 4.25
    assert abs(bench.job_gbs(1, 1.08e9, 8.0) - 135.0) < 1e-9


def _reference_arm(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", str(world), "--steps", "1", "--warmup", "0",
                           "--shape", "9,9,9"], env=env, capture_output=True, text=True,
                          timeout=300)


def test_reference_arm_runs_on_rank_zero_only(oracle):
    other = _reference_arm(1, 2)
    assert other.returncode == 0 and other.stdout.strip() == ""
    r0 = _reference_arm(0, 2)
    assert r0.returncode == 0, r0.stderr
    lines = [ln for ln in r0.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
