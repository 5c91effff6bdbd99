"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the job's
time is the slowest rank's and its converged count the sum over ranks; each
rank solves its own batch (weak scaling: generator seeds offset by rank); the
reference arm runs on rank 0 alone and prints one line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reduce_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, n = bench.reduce_over_ranks(torch, world, 10.0 + 5.0 * rank, 100 + rank, device="cpu")
        out[rank] = (ms, n)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_is_max_time_and_summed_count():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_reduce_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (15.0, 201)


def test_ranks_solve_different_batches():
    sys.path.insert(0, ROOT)
    from paper_2505_03728_gb300 import synth
    cfg = dict(synth.IK_THROUGHPUT, batch=64)
    per_rank = []
    for rank in range(2):
        c = dict(cfg, target_seed=cfg["target_seed"] + 1000 * rank, seed_seed=cfg["seed_seed"] + 1000 * rank)
        spec, qt, sd = synth.ik_workload(c)
        per_rank.append((qt, sd))
    assert not np.allclose(per_rank[0][0], per_rank[1][0])
    assert not np.allclose(per_rank[0][1], per_rank[1][1])


def test_reference_arm_prints_once_on_rank_zero():
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1")
        procs.append(subprocess.Popen([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                                       "--warmup", "0"], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    assert all(p.returncode == 0 for p in procs), [o[1][-500:] for o in outs]
    assert outs[1][0].strip() == ""
    line = json.loads(outs[0][0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_warmups_when_the_sample_covers_the_workload():
    """With a 64-target workload the calibrated per-step sample covers every
    target, so every warm-up and timed step must take the whole workload
    rather than slice past its end."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--batch", "64", "--steps", "2",
                        "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["warmup"] == 3 and line["steps"] == 2
    assert line["value"] > 0 and "64 targets" in line["cpu_baseline"]["sample"]
