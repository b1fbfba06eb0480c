"""The N > 1 path of the benchmark on CPU: two gloo ranks on 127.0.0.1.

The hot path does not shard (right-hand sides, chains and probes are
independent), so `bench.py --gpus N` runs one independent replica per rank
with its own seeded inputs and combines only the timing: the job's rate is
the units all ranks processed over the slowest rank's time. These tests run
that combination and the per-rank input draws with the gloo backend; no GPU
is involved."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    import holstein_inputs as hi
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 16 * (r + 1) units in 100 * (r + 1) ms
        units, ms = 16.0 * (rank + 1), 100.0 * (rank + 1)
        rate = bench.job_rate(world, units, ms, device="cpu")
        mx = bench.reduce_max(world, ms, device="cpu")
        sm = bench.reduce_sum(world, units, device="cpu")
        w = hi.WORKLOADS["tiny"]
        x, R = bench.replica_inputs(w, 2, rank)
        bench.barrier(world)
        out.put((rank, rate, mx, sm, float(x.sum()), float(R.sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    # every rank sees the same job figures: (16 + 32) units / max(100, 200) ms
    for rank, rate, mx, sm, _, _ in res:
        assert mx == 200.0 and sm == 48.0
        assert rate == pytest.approx(48.0 / 0.2)
    # the replicas draw different inputs
    assert res[0][4] != res[1][4] and res[0][5] != res[1][5]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(1, 32.0, 80.0) == pytest.approx(400.0)
    assert bench.reduce_max(1, 3.0) == 3.0 and bench.reduce_sum(1, 3.0) == 3.0


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun the oracle arm runs on rank 0 alone; another rank
    returns at once with status 0 and prints nothing."""
    import subprocess
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
