"""pk_ik_solve_split: the multi-start LM solve in two launches (every problem
up to a split iteration, then the suspended ones resumed from their saved
configuration, iteration count and damping).

A resumed problem recomputes its cost, Jacobian and normal matrix at the saved
configuration, which is exactly what the single launch holds there, so with
sibling cancellation off (each problem's iterates then depend on nothing but
its own inputs) the outputs equal pk_ik_solve's bit for bit.  With
cancellation on, when a sibling's convergence is seen depends on timing in
both paths; there the results are checked for validity.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_03728_gb300 import build, pk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def chain_case(B, S, n=7, seed=0, prismatic=()):
    spec = synth.chain_robot(9, n, prismatic=prismatic) if prismatic else synth.chain_robot(100, n)
    o = oracle.Robot.from_dict(spec)
    g = pk.Robot.from_spec(spec)
    ee = o.n_joints - 1
    qt = synth.uniform_q(900 + seed, B, o.dof_lower, o.dof_upper)
    targets = oracle.fk(o, qt)[:, ee:ee + 1]
    seeds = synth.uniform_q(950 + seed, (B, S), o.dof_lower, o.dof_upper)
    return o, g, [ee], None, dev(targets), dev(seeds)


def split_ws(g, B, S):
    return torch.zeros(pk.pk_ik_split_workspace_bytes(g, B, S), dtype=torch.uint8, device="cuda")


def records(g, ws, B, S):
    """The per-seed records of a split workspace: iteration counts and statuses."""
    n = g.n_dof
    stride = ((n + 3) & ~3) + 4
    off = 256 + ((B * 4 + 255) & ~255)
    rec = ws[off:off + B * S * stride * 4].view(torch.int32).view(B * S, stride)
    word = rec[:, stride - 1].cpu().numpy()
    return word & 0xFFFFFF, word >> 24


def same(a, b):
    for x, y in zip(a, b):
        assert torch.equal(x, y), (x - y).abs().max() if x.is_floating_point() else (x != y).sum()


@pytest.mark.parametrize("split", [1, 3, 7, 29])
@pytest.mark.parametrize("tail_ctas", [0, 2])
def test_split_equals_single_launch_without_cancellation(split, tail_ctas):
    B, S = 1500, 8
    o, g, links, kinds, targets, seeds = chain_case(B, S)
    p = pk.pk_ik_params_default(max_iters=30, early_exit=1, cancel_siblings=0)
    ref = pk.pk_ik_solve(g, p, links, kinds, targets, seeds)
    ws = split_ws(g, B, S)
    side = torch.cuda.Stream()
    got = pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, ws, split, tail_ctas, tail_stream=side)
    side.synchronize()
    same(got, ref)
    # every problem that ran past the split was suspended exactly once
    it, st = records(g, ws, B, S)
    n_resumed = int(ws[128:132].view(torch.int32).item())
    assert n_resumed == int((it > split).sum())
    assert not np.any(st == 15)  # no record is left suspended
    if split < 29:
        assert n_resumed > 0
    # the two launches' work adds up to the single launch's
    ws1 = torch.zeros(pk.pk_ik_workspace_bytes(g, B, S), dtype=torch.uint8, device="cuda")
    pk.pk_ik_solve(g, p, links, kinds, targets, seeds, ws1)
    one = pk.pk_ik_workspace_stats(ws1)
    first, second = pk.pk_ik_split_workspace_stats(ws)
    assert second["problems"] == n_resumed and first["problems"] + second["problems"] == B * S == one["problems"]
    # a resumed problem re-evaluates once at its saved configuration, and
    # rebuilds there unless the single launch did so anyway (last step accepted)
    assert first["evals"] + second["evals"] == one["evals"] + n_resumed
    assert one["builds"] <= first["builds"] + second["builds"] <= one["builds"] + n_resumed
    assert first["solves"] + second["solves"] == one["solves"]


def test_split_on_one_stream_and_the_general_chain_kernel():
    # prismatic joints take the general (non-fast) chain kernel
    B, S = 700, 4
    o, g, links, kinds, targets, seeds = chain_case(B, S, n=6, prismatic=(0, 3))
    p = pk.pk_ik_params_default(max_iters=25, early_exit=1, cancel_siblings=0)
    ref = pk.pk_ik_solve(g, p, links, kinds, targets, seeds)
    got = pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, split_ws(g, B, S), 4, 1)
    torch.cuda.synchronize()
    same(got, ref)


def test_split_without_early_exit_runs_every_problem_to_the_cap():
    B, S = 300, 2
    o, g, links, kinds, targets, seeds = chain_case(B, S, seed=3)
    p = pk.pk_ik_params_default(max_iters=12, early_exit=0, cancel_siblings=0)
    ref = pk.pk_ik_solve(g, p, links, kinds, targets, seeds)
    ws = split_ws(g, B, S)
    got = pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, ws, 5, 3)
    torch.cuda.synchronize()
    same(got, ref)
    assert int(ws[128:132].view(torch.int32).item()) == B * S
    assert torch.all(got[2] == 12)


def test_split_with_cancellation_is_valid():
    B, S = 4000, 8
    o, g, links, kinds, targets, seeds = chain_case(B, S, seed=5)
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=1)
    ref = pk.pk_ik_solve(g, p, links, kinds, targets, seeds)
    side = torch.cuda.Stream()
    q, err, iters, status = pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, split_ws(g, B, S), 6, 4,
                                                 tail_stream=side)
    side.synchronize()
    conv = status.cpu().numpy() == pk.PK_P_CONVERGED
    conv_ref = ref[3].cpu().numpy() == pk.PK_P_CONVERGED
    assert abs(conv.mean() - conv_ref.mean()) <= 0.01, (conv.mean(), conv_ref.mean())
    # converged answers meet the tolerance when re-checked in FP64
    qh = q.cpu().numpy().astype(np.float64)[conv]
    T = oracle.fk(o, qh)[:, links[0]].reshape(-1, 12)
    tg = targets.cpu().numpy().astype(np.float64)[conv, 0]
    pos = np.linalg.norm(T[:, [3, 7, 11]] - tg[:, [3, 7, 11]], axis=1)
    assert pos.max() <= p.tol_pos * 1.01
    e = err.cpu().numpy()[conv]
    assert np.all(e[:, 0] <= p.tol_pos) and np.all(e[:, 1] <= p.tol_rot)
    assert np.all(iters.cpu().numpy() <= 50)


def test_split_on_a_tree_robot_is_one_launch():
    spec, links = synth.humanoid_robot(103)
    o = oracle.Robot.from_dict(spec)
    g = pk.Robot.from_spec(spec)
    B, S = 64, 2
    qt = synth.uniform_q(40, B, o.dof_lower, o.dof_upper)
    targets = dev(oracle.fk(o, qt)[:, list(links)])
    seeds = dev(synth.uniform_q(41, (B, S), o.dof_lower, o.dof_upper))
    p = pk.pk_ik_params_default(max_iters=20, early_exit=1, cancel_siblings=0)
    ref = pk.pk_ik_solve(g, p, list(links), None, targets, seeds)
    side = torch.cuda.Stream()
    got = pk.pk_ik_solve_split(g, p, list(links), None, targets, seeds, split_ws(g, B, S), 3, 2, tail_stream=side)
    side.synchronize()
    same(got, ref)


def test_split_graph_capture_with_a_forked_tail():
    B, S = 1000, 8
    o, g, links, kinds, targets, seeds = chain_case(B, S, seed=7)
    p = pk.pk_ik_params_default(max_iters=30, early_exit=1, cancel_siblings=0)
    ref = pk.pk_ik_solve(g, p, links, kinds, targets, seeds)
    ws = split_ws(g, B, S)
    out = tuple(torch.empty_like(x) for x in ref)
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    s0 = torch.cuda.Stream()
    with torch.cuda.stream(s0):
        with torch.cuda.graph(graph, stream=s0):
            side.wait_stream(s0)
            pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, ws, 4, 2, out=out, stream=s0, tail_stream=side)
            s0.wait_stream(side)
    for _ in range(2):
        for x in out:
            x.zero_()
        graph.replay()
        torch.cuda.synchronize()
        same(out, ref)


def test_split_argument_checks():
    B, S = 10, 2
    o, g, links, kinds, targets, seeds = chain_case(B, S)
    p = pk.pk_ik_params_default()
    ws = split_ws(g, B, S)
    with pytest.raises(pk.PkError):
        pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, ws, 0)
    with pytest.raises(pk.PkError):
        pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, ws, 3, -1)
    small = torch.zeros(pk.pk_ik_workspace_bytes(g, B, S), dtype=torch.uint8, device="cuda")
    with pytest.raises(pk.PkError):
        pk.pk_ik_solve_split(g, p, links, kinds, targets, seeds, small, 3)
    assert pk.pk_ik_split_workspace_bytes(g, B, S) > pk.pk_ik_workspace_bytes(g, B, S)


def test_full_size_split_equals_single_launch_without_cancellation():
    """The throughput workload at full size (65,536 targets x 8 seeds, up to 50
    iterations) through the split solve in the bench's launch configuration
    (first launch up to 8 iterations, 24-block continuation on a second
    stream): bit-identical to the single launch when siblings do not cancel."""
    cfg = synth.IK_THROUGHPUT
    spec, qt, sd = synth.ik_workload(cfg)
    g = pk.Robot.from_spec(spec)
    ee = g.n_joints - 1
    targets = pk.pk_fk(g, dev(qt))[:, ee:ee + 1].contiguous()
    seeds = dev(sd)
    B, S = sd.shape[0], sd.shape[1]
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    ref = pk.pk_ik_solve(g, p, [ee], None, targets, seeds)
    side = torch.cuda.Stream()
    got = pk.pk_ik_solve_split(g, p, [ee], None, targets, seeds, split_ws(g, B, S), 8, 24, tail_stream=side)
    side.synchronize()
    same(got, ref)


def test_full_size_pipelined_learned_steps_are_valid():
    """Consecutive learned-seed steps overlapped as the bench runs them (seed
    inference and first launch on one stream, continuation and selection on a
    second, two workspaces, a different target batch per step, sibling
    cancellation on): every step's converged answers meet the tolerance when
    re-checked in FP64, and the success rate matches one batch at a time."""
    cfg = synth.IK_THROUGHPUT
    spec, qt, sd = synth.ik_workload(cfg)
    g, o = pk.Robot.from_spec(spec), oracle.Robot.from_dict(spec)
    ee = g.n_joints - 1
    B, S, n = sd.shape
    net = pk.SeedNet(g, [ee], K=S, width=512, depth=4, seed=11)
    pk.pk_seednet_train(net, pk.pk_train_params_default(epochs=2, steps_per_epoch=600, batch=8192, seed=500))
    steps = 3
    qts = [qt] + [synth.uniform_q(77 + k, B, o.dof_lower, o.dof_upper) for k in range(1, steps)]
    T = [pk.pk_fk(g, dev(q))[:, ee:ee + 1].contiguous() for q in qts]
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=1)
    wss = [split_ws(g, B, S) for _ in range(2)]
    lseeds = torch.empty(B, S, n, device="cuda")
    outs = [tuple(torch.empty(B, *shape, device="cuda", dtype=dt) for shape, dt in
                  (((n,), torch.float32), ((2,), torch.float32), ((), torch.int32), ((), torch.int32)))
            for _ in range(steps)]
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    done = [torch.cuda.Event() for _ in range(steps)]
    for k in range(steps):
        if k >= 2:
            main.wait_event(done[k - 2])
        pk.pk_seednet_infer(net, T[k], lseeds, stream=main)
        pk.pk_ik_solve_split(g, p, [ee], None, T[k], lseeds, wss[k % 2], 8, 24, out=outs[k], stream=main,
                             tail_stream=side)
        done[k].record(side)
    torch.cuda.synchronize()
    tg = oracle.Targets([ee])
    for k in range(steps):
        q, err, iters, status = [x.cpu().numpy() for x in outs[k]]
        conv = status == pk.PK_P_CONVERGED
        # one batch at a time, single launch
        ref_status = pk.pk_ik_solve(g, p, [ee], None, T[k], pk.pk_seednet_infer(net, T[k]))[3].cpu().numpy()
        assert abs(conv.mean() - (ref_status == 0).mean()) <= 0.002, (k, conv.mean(), (ref_status == 0).mean())
        assert conv.mean() >= 0.9
        targets = T[k].cpu().numpy().astype(np.float64)
        idx = np.nonzero(conv)[0]
        for b in np.random.default_rng(k).choice(idx, 500, replace=False):
            pe, re = oracle.ik_errors(o, tg, targets[b], q[b].astype(np.float64))
            assert pe <= p.tol_pos * (1 + 1e-3) and re <= p.tol_rot * (1 + 1e-3)
        assert np.all(iters <= 50)
