"""Uneven batches: one persistent launch over a 6-DoF chain, a 7-DoF chain, the
24-DoF hand (five position targets) and the 30-joint humanoid (six pose
targets), replayed as a CUDA graph, with an autotuned schedule.

Checks: graph replay equals the eager launch sequence bit for bit; the plan's
per-robot results match separate pk_ik_solve calls (same statuses, q within
1e-5 relative where both converged); after autotuning (which may move the
chains to the warp-per-problem path and reorder the sets) the solved set is
unchanged up to FP32 schedule effects (>= 97% identical statuses) and every
converged solution passes the FP64 oracle check."""
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


def make(scale):
    sets, meta = [], []
    for name, spec, links, kinds, qt, sd in synth.uneven_workload(scale=scale):
        g = pk.Robot.from_spec(spec)
        T = pk.pk_fk(g, dev(qt))[:, links].contiguous()
        sets.append((g, links, kinds, T, dev(sd)))
        meta.append((name, spec, links, kinds))
    return sets, meta


def host(outs):
    return [[x.cpu().numpy() for x in o] for o in outs]


def test_graph_equals_eager_and_matches_single_solves():
    sets, meta = make(0.05)
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    plan = pk.IkPlan(p, sets)
    eager = host(plan.run(graph=False))
    graph = host(plan.run(graph=True))
    for a, b in zip(eager, graph):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
    for (g, links, kinds, T, sd), (q, err, it, st) in zip(sets, graph):
        q1, e1, i1, s1 = [x.cpu().numpy() for x in pk.pk_ik_solve(g, p, links, kinds, T, sd)]
        np.testing.assert_array_equal(st, s1)
        both = (st == 0) & (s1 == 0)
        np.testing.assert_allclose(q[both], q1[both], rtol=1e-5, atol=1e-5)


def test_autotuned_schedule_keeps_results_valid():
    sets, meta = make(0.05)
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=1)
    plan = pk.IkPlan(p, sets)
    base = host(plan.run())
    ms = plan.autotune(reps=2)
    sched = plan.schedule()
    assert ms > 0 and sched["block"] in (64, 128, 256)
    tuned = host(plan.run())
    for (name, spec, links, kinds), (g, _, _, T, sd), a, b in zip(meta, sets, base, tuned):
        assert (a[3] == b[3]).mean() >= 0.97, name
        o = oracle.Robot.from_dict(spec)
        tg = oracle.Targets(links, kinds)
        Th = T.cpu().numpy()
        for i in np.nonzero(b[3] == 0)[0]:
            pe, re = oracle.ik_errors(o, tg, Th[i], b[0][i])
            assert pe <= 1e-3 * (1 + 1e-3) and re <= np.deg2rad(0.5) * (1 + 1e-3), name
    # every schedule is valid: each variant, the other chain path, the given order
    for variant in range(4):
        plan.set_schedule(block=64, chains_as_trees=1 - sched["chains_as_trees"], given_order=1,
                          variant=variant)
        other = host(plan.run())
        for a, b in zip(base, other):
            assert (a[3] == b[3]).mean() >= 0.97, variant
    st = plan.stats()
    assert st["problems"] > 0


def test_persistent_launch_without_chain_path_matches_specialised_kernels():
    """With every set on the warp path (chains_as_trees = 1) the single
    persistent launch (variants 0 and 1) is the instantiation without the
    thread-per-problem chain path; without sibling cancellation its results
    match the specialised tree kernels' on the same path (variant 2)."""
    sets, meta = make(0.05)
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    plan = pk.IkPlan(p, sets)
    plan.set_schedule(block=128, chains_as_trees=1, given_order=1, variant=2)
    ref = host(plan.run())
    for variant, block in ((0, 64), (0, 256), (1, 128)):
        plan.set_schedule(block=block, chains_as_trees=1, given_order=1, variant=variant)
        got = host(plan.run())
        for (name, *_), (q0, _, _, s0), (q1, _, _, s1) in zip(meta, ref, got):
            np.testing.assert_array_equal(s1, s0, err_msg=f"{name} variant {variant} block {block}")
            both = s0 == 0
            np.testing.assert_allclose(q1[both], q0[both], rtol=1e-5, atol=1e-5)
