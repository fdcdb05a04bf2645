"""Host logic of multi-GPU replica runs, exercised as two gloo ranks on the CPU:
the job's time is the slowest rank's, its work the sum over ranks, and no two
ranks share a Philox chain id."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as tmp

from paper_0903_3053_gb300 import replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        replicas.barrier(world)
        secs = [2.0, 3.5][rank]
        units = [100.0, 50.0][rank]
        res = {
            "max": replicas.max_over_ranks(secs, world, "cpu"),
            "sum": replicas.sum_over_ranks(units, world, "cpu"),
            "rate": replicas.job_rate(units, secs, world, "cpu"),
            "ids": [replicas.chain_id(rank, i) for i in range(20)],
        }
        gathered = [None] * world
        dist.all_gather_object(gathered, res)
        if rank == 0:
            out.put(gathered)
        replicas.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g["max"] for g in got] == [3.5, 3.5]
    assert [g["sum"] for g in got] == [150.0, 150.0]
    assert got[0]["rate"] == pytest.approx(150.0 / 3.5)
    assert not set(got[0]["ids"]) & set(got[1]["ids"])


def test_chain_id_ranges():
    assert replicas.chain_id(0, 5) == 5
    assert replicas.chain_id(3, 0) == 3 * replicas.CHAIN_ID_STRIDE
    with pytest.raises(ValueError):
        replicas.chain_id(0, replicas.CHAIN_ID_STRIDE)
    with pytest.raises(ValueError):
        replicas.chain_id(1 << 16, 0)


def test_single_rank_is_identity():
    assert replicas.max_over_ranks(1.25, 1) == 1.25
    assert replicas.job_rate(10.0, 2.0, 1) == 5.0


def test_reference_arm_on_nonzero_rank_does_no_work():
    """Under torchrun only rank 0 runs the reference arm; the others exit 0
    silently."""
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_json_line():
    """The reference arm (the CPU oracle on a bounded sample of the benchmark
    workload) prints one JSON line with the contract's keys."""
    import json
    env = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
