"""The multi-rank side of bench.py on CPU (gloo, world size 2): the timed region is the
slowest rank's, the value counts every rank's batch (weak scaling), ranks draw independent
fields, and the reference arm prints from rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")


def _worker(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 1.0 + rank                       # rank 1 is the slower one
        t = bench._max_over_ranks(elapsed, dist, "cpu")
        v = bench._weak_value(2_000_000, 10, world, t)
        out_q.put((rank, t, v, bench._rank_seed(rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_weak_value_gloo():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, v0, s0), (r1, t1, v1, s1) = res
    assert t0 == t1 == 2.0                         # max over ranks, same on every rank
    assert v0 == v1 == pytest.approx(2_000_000 * 10 * 2 / 2.0 / 1e9)
    assert s0 != s1                                # independent load cases per rank


def test_single_rank_helpers():
    import bench
    assert bench._max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench._weak_value(1e9, 1, 1, 1.0) == pytest.approx(1.0)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GDOF/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_recorded_traffic_belongs_to_the_current_kernel_sources():
    """The DRAM traffic bench.py reports was captured on the kernel sources whose
    hash it records; a change to those sources without a new capture must show
    up here (bench.py then reports traffic as null)."""
    import bench
    assert bench.TRAFFIC["bytes_per_field"] > 0
    assert bench._src_hash(bench.TRAFFIC["sources"]) == bench.TRAFFIC["sha256"]
