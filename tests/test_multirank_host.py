"""The multi-rank host logic of bench.py on CPU: two gloo ranks launched the way torchrun
launches them (RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT in the environment).

Several GPUs run independent replicas of the step (no data-path collective): the only
cross-rank steps are the barriers around the timed region and the max over the ranks'
timed regions, and the whole-job value counts the units of every rank.  The reference
(oracle) arm and the single-GPU workloads run on rank 0 alone; the other ranks exit 0
without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["PAWFD_ROOT"])
import torch
import torch.distributed as dist
import bench
world, rank, local = bench.dist_env()
dist.init_process_group("gloo")
dist.barrier()
mine = [0.40, 0.65][rank]
job = bench.max_over_ranks(mine, world, torch.device("cpu"))
value = bench.job_throughput(2.0e9, world, job)
dist.barrier()
print(json.dumps({"rank": rank, "world": world, "local": local, "job": job, "value": value}), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def launch(args, world, extra_env=None, timeout=120):
    port = free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), PAWFD_ROOT=ROOT, **(extra_env or {}))
        procs.append(subprocess.Popen([sys.executable] + args, cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    try:
        for p in procs:
            out, err = p.communicate(timeout=timeout)
            outs.append((p.returncode, out, err))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    return outs


def test_two_gloo_ranks_take_the_max_time_and_count_every_rank():
    outs = launch(["-c", WORKER], 2)
    for rc, out, err in outs:
        assert rc == 0, err[-2000:]
    recs = sorted((json.loads(out.strip().splitlines()[-1]) for _, out, _ in outs), key=lambda r: r["rank"])
    assert [r["rank"] for r in recs] == [0, 1] and all(r["world"] == 2 for r in recs)
    assert [r["local"] for r in recs] == [0, 1]
    # both ranks see the slower rank's time, and the value counts both ranks' units
    assert all(r["job"] == pytest.approx(0.65, rel=0, abs=1e-15) for r in recs)
    assert all(r["value"] == pytest.approx(2 * 2.0 / 0.65, rel=1e-15) for r in recs)


def test_one_rank_is_the_identity():
    import bench
    assert bench.max_over_ranks(0.123, 1, None) == 0.123
    assert bench.job_throughput(5.0e9, 1, 2.0) == pytest.approx(2.5)


def rank_one(args):
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT="1")
    return subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=120)


def test_reference_arm_runs_on_rank_zero_only():
    # rank 1 returns before building or running the oracle: no output, exit 0
    r = rank_one(["--impl", "reference"])
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("workload", ["served", "davidson", "density", "poisson"])
def test_single_gpu_workloads_skip_the_other_ranks(workload):
    r = rank_one(["--workload", workload])
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
