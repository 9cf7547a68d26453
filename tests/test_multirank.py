"""Host logic of the multi-GPU benchmark path, on CPU with the gloo backend (2 ranks).

Each rank simulates its own batch of independent worlds (no data-path collective); the
timings are max-reduced and the agent counts summed, and rank 0 alone reports.  The
reference arm (the CPU oracle) runs on rank 0 only; other ranks exit without work.
"""
import hashlib
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import worldgen as wg
        wl = bench.rank_workload(wg.WORKLOADS["tiny"], rank)
        worlds = wg.make_workload(wl)
        digest = hashlib.sha256(np.ascontiguousarray(worlds.boxes).tobytes() +
                                np.ascontiguousarray(worlds.road).tobytes()).hexdigest()
        digests = [None] * world
        dist.all_gather_object(digests, digest)
        my_ms = 10.0 + 5.0 * rank  # a rank-dependent "measured" time
        max_ms = bench.reduce_over_ranks(my_ms, "max", world, "cpu")
        total_agents = bench.reduce_over_ranks(worlds.n_agents + rank, "sum", world, "cpu")
        rate = bench.job_rate(total_agents, 4, max_ms)
        q.put((rank, wl.seed, digests, max_ms, total_agents, rate, worlds.n_agents))
    finally:
        dist.destroy_process_group()


def test_two_ranks_independent_batches_and_reductions():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seed0, dig0, max0, tot0, rate0, n0), (r1, seed1, dig1, max1, tot1, rate1, n1) = res
    assert seed0 != seed1
    assert dig0 == dig1 and dig0[0] != dig0[1]  # each rank built its own, different worlds
    assert max0 == max1 == 15.0  # slowest rank's time
    assert tot0 == tot1 == n0 + n1 + 1  # every rank's agents
    assert rate0 == rate1 == pytest.approx((n0 + n1 + 1) * 4 / 0.015)


def _bench(env_extra, args):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, env=env,
                          capture_output=True, text=True, timeout=300, cwd=ROOT)


def test_reference_arm_nonzero_rank_exits_without_work():
    r = _bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"},
               ["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_rank0_prints_one_line():
    r = _bench({"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0", "GP_REF_STEP_SECONDS": "0.3"},
               ["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle"
    # the oracle runs on every host core, one process each
    assert d["cpu_baseline"]["cores"] == (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                                          else os.cpu_count())
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
