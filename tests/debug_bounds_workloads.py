"""Small workloads of every kernel family that carries index checks, run
against the library that PK_DEBUG_BOUNDS selects (1: the checked build
libpk_debug.so, otherwise libpk.so).  Writes each workload's outputs and, in
the checked build, the status word read after it to the .npz given as the
first argument.  tests/test_gpu_debug_bounds.py runs it once per library in
a subprocess and compares the two files.

Sibling cancellation is off so that every output is deterministic.
"""
import sys

import numpy as np
import torch

from paper_2505_03728_gb300 import pk, scenes, synth


def main(out_path):
    res = {}
    checked = pk.pk_debug_bounds_enabled()
    res["checked"] = np.array(int(checked))
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")

    def keep(name, outs):
        torch.cuda.synchronize()
        for i, o in enumerate(outs):
            res[f"{name}_{i}"] = o.detach().cpu().numpy()
        if checked:
            res[f"bounds_{name}"] = np.array(pk.pk_debug_bounds_take(), dtype=np.uint64)

    # chain: single launch, split launch (the continuation claims resumed
    # records), best-seed selection, then the collision-free choice
    spec = synth.chain_robot(100, 7)
    g = pk.Robot.from_spec(spec)
    ee = g.n_joints - 1
    B, S = 256, 8
    qt = synth.uniform_q(11, B, spec.dof_lower, spec.dof_upper)
    sd = dev(synth.uniform_q(12, (B, S), spec.dof_lower, spec.dof_upper))
    T = pk.pk_fk(g, dev(qt))[:, ee:ee + 1].contiguous()
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    ws = torch.empty(pk.pk_ik_workspace_bytes(g, B, S), dtype=torch.uint8, device="cuda")
    out = pk.pk_ik_solve(g, p, [ee], None, T, sd, ws)
    keep("chain", out)
    wss = torch.empty(pk.pk_ik_split_workspace_bytes(g, B, S), dtype=torch.uint8, device="cuda")
    keep("split", pk.pk_ik_solve_split(g, p, [ee], None, T, sd, wss, 4, 8))
    cfg = synth.TRAJOPT
    tspec, qs_c, qg_c, radii, obs, plane = synth.trajopt_workload(cfg)
    pk.pk_ik_select_clear(g, ws, S, dev(radii), dev(obs), plane, 0.02, out=out)
    keep("select_clear", out)

    # IK-Beam (kept-seed gather)
    beam = pk.pk_ik_beam_params_default()
    Bb = 16
    sb = dev(synth.uniform_q(13, (Bb, beam.n_seeds), spec.dof_lower, spec.dof_upper))
    keep("beam", pk.pk_ik_beam_solve(g, p, beam, [ee], None, T[:Bb].contiguous(), sb))

    # tree: the humanoid (level lists, parents, variables, target links)
    hspec, ends = synth.humanoid_robot(103)
    h = pk.Robot.from_spec(hspec)
    links = list(ends)
    Bh, Sh = 64, 4
    qh = synth.uniform_q(14, Bh, hspec.dof_lower, hspec.dof_upper)
    Th = pk.pk_fk(h, dev(qh))[:, links].contiguous()
    sh = dev(synth.uniform_q(15, (Bh, Sh), hspec.dof_lower, hspec.dof_upper))
    keep("tree", pk.pk_ik_solve(h, p, links, None, Th, sh))

    # trajectories (obstacle screening), the first 8 of the workload
    tg = pk.Robot.from_spec(tspec)
    pts = lambda q: pk.pk_fk(tg, dev(q)).cpu().numpy()[:, :, [3, 7, 11]].astype(np.float64)
    Bt = 8
    qs = scenes.pick_clear(qs_c[:256], pts(qs_c[:256]), radii, obs, plane, 0.02, Bt)
    qg = scenes.pick_clear(qg_c[:256], pts(qg_c[:256]), radii, obs, plane, 0.02, Bt)
    goals = pk.pk_fk(tg, dev(qg))[:, -1].contiguous()
    x0 = dev(synth.linear_interpolation(qs, qg, cfg["T"]))
    tp = pk.pk_trajopt_params_default(iters=20)
    keep("trajopt", pk.pk_trajopt_solve(tg, tp, dev(qs), goals, x0, dev(radii), dev(obs), plane))

    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
