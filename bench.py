"""Benchmark: converged IK solves per second on one GB300 (or N, weak scaling).

Workload (default): the throughput IK workload -- a seeded synthetic 7-DoF
revolute chain, 65,536 reachable target poses (FK of uniform in-limit
configurations), 8 uniform random seeds per target (524,288 LM problems), up
to 50 LM iterations with early exit at 1 mm / 0.5 deg, and sibling
cancellation (a target stops once one of its seeds converged).  One step =
one pk_ik_solve of the whole batch with inputs resident in HBM; every timed
step is preceded by an L2 flush (a 256 MiB device write outside the timed
events).  value = converged targets / device time.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pk|reference]
Multi-GPU: launched by torchrun, one rank per GPU; every rank solves its own
65,536-target batch (different generator seeds), no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "converged IK solves/s at ≤1mm/0.5° (learned-seed vs plain LM, 1 GB300)"
UNIT = "solves/s"

# FP32 operations (add, mul = 1; fma = 2) per unit of work of the fused LM
# kernel for the 7-DoF chain, from ncu's per-thread executed FADD/FMUL/FFMA
# counts over launches with known work counters (see profiles/).
FLOPS_PER_EVAL = 1207.4
FLOPS_PER_BUILD = 1362.0
FLOPS_PER_SOLVE = 172.4
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12  # SMs x FP32 lanes x 2 x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["pk", "reference"], default="pk")
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--no-cancel", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(spec, qt, sd, n_targets, max_iters=50):
    """The FP64 oracle (as it stands) on the first n_targets targets of the
    workload, all host cores; returns (converged, seconds, threads)."""
    import oracle
    o = oracle.Robot.from_dict(spec)
    ee = o.n_joints - 1
    targets = oracle.fk(o, qt[:n_targets])[:, [ee]]
    prm = oracle.IkParams(max_iters=max_iters, early_exit=1)
    t0 = time.perf_counter()
    out = oracle.ik_solve(o, prm, oracle.Targets([ee]), targets, sd[:n_targets])
    dt = time.perf_counter() - t0
    return int(np.sum(out["status"] == 0)), dt, out["threads"]


def cpu_baseline(spec, qt, sd, budget_s=12.0):
    conv, dt, thr = oracle_sample(spec, qt, sd, 64)
    n = int(min(len(qt), max(64, 64 * budget_s / max(dt, 1e-3))))
    conv, dt, thr = oracle_sample(spec, qt, sd, n)
    return {"value": conv / dt, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": f"first {n} targets x {sd.shape[1]} seeds of the workload, FP64, "
                      f"{dt:.1f} s wall on {thr} threads ({conv}/{n} converged)"}


def run_reference(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2505_03728_gb300 import synth
    spec, qt, sd = synth.ik_workload(cfg)
    # calibrate a per-step sample of ~3 s
    conv, dt, thr = oracle_sample(spec, qt, sd, 32)
    n = int(min(len(qt), max(32, 32 * 3.0 / max(dt, 1e-3))))
    for w in range(args.warmup):
        oracle_sample(spec, qt[w * n:], sd[w * n:], n)
    tot_c, tot_t = 0, 0.0
    for k in range(args.steps):
        off = (k * n) % max(1, len(qt) - n)
        c, t, thr = oracle_sample(spec, qt[off:], sd[off:], n)
        tot_c += c
        tot_t += t
    value = tot_c / tot_t
    sample = f"{n} targets x {sd.shape[1]} seeds per step (of {len(qt)}), FP64 on {thr} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(cfg, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def config_dict(cfg, args):
    return {"workload": cfg["name"], "robot": "synthetic 7-DoF revolute chain (seed 100)",
            "targets": args.batch, "seeds_per_target": cfg["n_seeds"], "max_iters": cfg["max_iters"],
            "early_exit": True, "cancel_siblings": not args.no_cancel, "seeding": "uniform random",
            "l2": "flushed by a 256 MiB device write before every timed step"}


# ----------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    from paper_2505_03728_gb300 import synth
    cfg = dict(synth.IK_THROUGHPUT)
    cfg["batch"] = args.batch
    if args.impl == "reference":
        run_reference(args, cfg)
        return

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2505_03728_gb300 import build, pk
    build.build()

    cfg_r = dict(cfg, target_seed=cfg["target_seed"] + 1000 * rank, seed_seed=cfg["seed_seed"] + 1000 * rank)
    spec, qt, sd = synth.ik_workload(cfg_r)
    robot = pk.Robot.from_spec(spec)
    ee = robot.n_joints - 1
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    B, S, n = sd.shape
    targets = pk.pk_fk(robot, dev(qt))[:, ee:ee + 1].contiguous()
    seeds = dev(sd)
    params = pk.pk_ik_params_default(max_iters=cfg["max_iters"], early_exit=1,
                                     cancel_siblings=0 if args.no_cancel else 1)
    ws = torch.empty(pk.pk_ik_workspace_bytes(robot, B, S), dtype=torch.uint8, device="cuda")
    outs = (torch.empty(B, n, device="cuda"), torch.empty(B, 2, device="cuda"),
            torch.empty(B, dtype=torch.int32, device="cuda"), torch.empty(B, dtype=torch.int32, device="cuda"))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        return pk.pk_ik_solve(robot, params, [ee], None, targets, seeds, ws, out=outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    conv = torch.zeros((), dtype=torch.int64, device="cuda")
    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    pk.pk_trace_enable(True)
    with ClockSampler(gpu_id) as clocks:
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
            conv += (outs[3] == pk.PK_P_CONVERGED).sum()
        torch.cuda.synchronize()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    lm_ms, lm_n = pk.pk_trace_summary("ik_lm")
    red_ms, red_n = pk.pk_trace_summary("ik_reduce")
    pk.pk_trace_enable(False)
    stats = pk.pk_ik_workspace_stats(ws)
    total_ms = float(sum(step_ms))
    n_conv = int(conv.item())
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = torch.tensor([n_conv], dtype=torch.int64, device="cuda")
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        total_ms, n_conv = float(t.item()), int(c.item())
    value = n_conv / (total_ms / 1e3)

    # end to end through the public API with host buffers
    h_t = torch.empty(targets.shape, dtype=torch.float32, pin_memory=True)
    h_t.copy_(targets)
    h_s = torch.empty(seeds.shape, dtype=torch.float32, pin_memory=True)
    h_s.copy_(seeds)
    h_out = [torch.empty(o.shape, dtype=o.dtype, pin_memory=True) for o in outs]
    d_t, d_s = torch.empty_like(targets), torch.empty_like(seeds)
    e2e_conv, e2e_ms = 0, 0.0
    for k in range(max(2, args.steps // 2) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d_t.copy_(h_t, non_blocking=True)
        d_s.copy_(h_s, non_blocking=True)
        pk.pk_ik_solve(robot, params, [ee], None, d_t, d_s, ws, out=outs)
        for ho, o in zip(h_out, outs):
            ho.copy_(o, non_blocking=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if k > 0:  # first one is a warm-up of the copies
            e2e_ms += dt * 1e3
            e2e_conv += int((h_out[3] == pk.PK_P_CONVERGED).sum())
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = torch.tensor([e2e_conv], dtype=torch.int64, device="cuda")
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        e2e_ms, e2e_conv = float(t.item()), int(c.item())
    h2d = h_t.numel() * 4 + h_s.numel() * 4
    d2h = sum(o.numel() * o.element_size() for o in outs)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    flops = (stats["evals"] * FLOPS_PER_EVAL + stats["builds"] * FLOPS_PER_BUILD
             + stats["solves"] * FLOPS_PER_SOLVE)
    lm_avg_ms = lm_ms / max(1, lm_n)
    achieved = flops / (lm_avg_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(cfg, args),
        "success_rate": n_conv / (B * args.steps * world),
        "roofline": {"bound": "alu", "kernel": "chain_lm_kernel<7>", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "traffic": None,
                     "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz (unit counts x max clock)",
                     "lm_kernel_ms": lm_avg_ms, "reduce_kernel_ms": red_ms / max(1, red_n),
                     "work_per_launch": stats},
        "e2e": {"value": e2e_conv / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, qt, sd)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
