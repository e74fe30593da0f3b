"""Host logic of `bench.py --gpus N`: N independent replicas, one per rank,
no data-path collective; the slowest rank's time and the units of all ranks
make the whole-job value.  Run here as two gloo ranks on CPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        mx = bench.max_over_ranks(local_ms)
        value = bench.replica_throughput(1000.0, world, mx)
        out.put((rank, mx, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_throughput_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, value in got:
        assert mx == 150.0  # every rank sees the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 0.150)


def test_single_process_aggregation_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.replica_throughput(10.0, 1, 1000.0) == 10.0


def _reference_arm(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", OMP_NUM_THREADS="2")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
                           "--steps", "1", "--warmup", "3", "--gpus", "2"],
                          env=env, capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_on_rank_zero_only():
    r1 = _reference_arm(1)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference_arm(0)
    assert r0.returncode == 0, r0.stderr
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
