"""Host logic of bench.py without a GPU.

* Replicas (the multi-GPU mode: each rank solves its own forcings, no data
  collective): with two gloo ranks on CPU the timing aggregation takes the
  slowest rank and the throughput counts every rank's solves.
* The reference arm (--impl reference) runs the FP64 oracle on the small
  16x16 workload and prints one JSON line with the contract's keys; a rank
  other than 0 prints nothing and exits 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [100.0, 150.0][rank]
    slowest = bench.max_over_ranks(ms, dist, device="cpu")
    q.put((rank, slowest, bench.throughput(world, 5, 2, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_takes_slowest_rank_and_counts_all_solves():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, value in out:
        assert slowest == 150.0
        assert abs(value - 2 * 5 * 2 / 0.150) < 1e-9


def test_throughput_without_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert abs(bench.throughput(1, 10, 1, 2000.0) - 5.0) < 1e-12


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "2d16",
                        "--steps", "2", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    # other ranks of a torchrun launch do no work
    env.update(RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "2d16",
                        "--steps", "2", "--warmup", "3"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
