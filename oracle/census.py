"""Algorithmic FLOPs of the hot path, counted on the oracle's own arithmetic.

TEST AND MEASUREMENT INFRASTRUCTURE ONLY.  ``python -m oracle.census``
prints the per-unit work that the benchmark's roofline lines multiply by the
GPU's live work counters (the benchmark carries the printed figures as
constants, and ``tests/test_flop_census.py`` checks that they still match).

The counting rule is that of ``flopcount.hpp``: +, -, *, / and sqrt are one
FLOP each, an operation with an exact-zero operand is structural and free,
sin / cos / atan2 / acos are counted apart, and the damped solves are counted
as the dense (banded) factorisations they are.  The work of a unit varies a
little with the state (which hinges are active, which collision pairs are
within eta, which series branch a small angle takes), so every figure is an
average over the states the oracle's own LM runs visit on the workload:

* IK, 7-DoF chain (the throughput workload): the seeds and every accepted
  iterate of oracle LM runs (50 iterations, early exit) on the first targets
  of the workload, 8 seeds each.  Units: a candidate evaluation (FK,
  residuals, cost), a build at an accepted point (Jacobian, J^T J, J^T r, the
  convergence errors) and a damped solve (Cholesky and both substitutions).
* Trajectories, 7-DoF chain, T = 64, 32 obstacles and the plane: the iterates
  of oracle LM runs (50 iterations) on the first trajectories of the
  workload.  Per trajectory-iteration the method evaluates one candidate and
  solves once; it builds the normal equations at accepted candidates, at the
  accept rate of those runs.
* Seed network: the multiply-adds of its layers, 2 x sum(in x out) per
  target, with the unpadded shapes (9 -> 512 -> 512 -> 512 -> 512 -> 8 x 7).
"""
from __future__ import annotations

import json
import sys

import numpy as np

import oracle
from paper_2505_03728_gb300 import scenes, synth


def ik_chain7(n_targets=16, n_seeds=8):
    cfg = synth.IK_THROUGHPUT
    spec, qt, sd = synth.ik_workload(cfg, n_targets)
    rb = oracle.Robot.from_dict(spec)
    ee = rb.n_joints - 1
    tg = oracle.Targets([ee])
    targets = oracle.fk(rb, qt)[:, [ee]]
    prm = oracle.IkParams(max_iters=cfg["max_iters"], early_exit=1)
    units = {"eval": [], "build": [], "solve": []}
    for b in range(n_targets):
        for s in range(n_seeds):
            o = oracle.lm_run(rb, prm, tg, targets[b], sd[b, s], cfg["max_iters"])
            states = [sd[b, s]] + [o["q_trace"][k] for k in range(o["iters"])]
            for q in states:
                u = oracle.ik_flop_units(rb, prm, tg, targets[b], q)
                for k in units:
                    units[k].append(u[k])
    out = {}
    for k, v in units.items():
        a = np.asarray(v, dtype=np.float64)
        out[k] = {"flops": float(a[:, 0].mean()), "special": float(a[:, 1].mean()),
                  "min": int(a[:, 0].min()), "max": int(a[:, 0].max())}
    out["states"] = len(units["eval"])
    return out


def trajopt7(n_traj=4):
    cfg = synth.TRAJOPT
    spec, qs_c, qg_c, radii, obs, plane = synth.trajopt_workload(cfg)
    rb = oracle.Robot.from_dict(spec)
    pts = lambda q: oracle.fk(rb, q)[:, :, [3, 7, 11]]
    cand = 64 * n_traj
    qs = scenes.pick_clear(qs_c[:cand], pts(qs_c[:cand]), radii, obs, plane, 0.02, n_traj)
    qg = scenes.pick_clear(qg_c[:cand], pts(qg_c[:cand]), radii, obs, plane, 0.02, n_traj)
    goals = oracle.fk(rb, qg)[:, -1]
    x0 = synth.linear_interpolation(qs, qg, cfg["T"])
    scene = oracle.Scene(radii, obs, plane)
    prm = oracle.TrajParams(iters=cfg["iters"])
    units = {"eval": [], "build": [], "solve": []}
    accepts = 0
    for b in range(n_traj):
        o = oracle.traj_lm_run(rb, prm, scene, x0[b], qs[b], goals[b])
        lam = np.concatenate([[prm.lambda0], o["lam_trace"]])
        accepts += int(np.sum(lam[1:] < lam[:-1]) + np.sum((lam[1:] == lam[:-1]) & (lam[1:] == prm.lambda_min)))
        for k in range(0, cfg["iters"], 7):
            x = x0[b] if k == 0 else o["trace"][k - 1]
            u = oracle.traj_flop_units(rb, prm, scene, x, qs[b], goals[b], lam=lam[k])
            for key in units:
                units[key].append(u[key])
    out = {}
    for k, v in units.items():
        a = np.asarray(v, dtype=np.float64)
        out[k] = {"flops": float(a[:, 0].mean()), "special": float(a[:, 1].mean()),
                  "min": int(a[:, 0].min()), "max": int(a[:, 0].max())}
    rate = accepts / (n_traj * cfg["iters"])
    out["accept_rate"] = rate
    out["flops_per_traj_iter"] = out["eval"]["flops"] + out["solve"]["flops"] + rate * out["build"]["flops"]
    out["flops_per_traj_init"] = out["eval"]["flops"] + out["build"]["flops"]
    out["T"], out["iters"], out["trajectories"] = cfg["T"], cfg["iters"], n_traj
    return out


def seednet7(width=512, depth=4, K=8, n=7, d_in=9):
    dims = [d_in] + [width] * depth + [K * n]
    return {"dims": dims, "flops_per_target": 2.0 * sum(a * b for a, b in zip(dims[:-1], dims[1:]))}


def census():
    return {"ik_chain7": ik_chain7(), "trajopt7_T64": trajopt7(), "seednet7": seednet7()}


if __name__ == "__main__":
    json.dump(census(), sys.stdout, indent=1)
    print()
