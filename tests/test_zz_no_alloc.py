"""pk_ik_solve_noalloc: the IK solve for callers that cannot allocate device
memory while they run (real-time loops, plugin hosts with their own
allocator).  Its scratch is the library's fixed 32 MiB device array; these
tests call it through the C ABI twice in a row and compare with pk_ik_solve,
which uses a caller workspace, and check the size limit.  This file is
collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2505_03728_gb300 import build, pk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


def _inputs(batch, seed_offset=0):
    cfg = dict(synth.IK_THROUGHPUT, target_seed=201 + seed_offset, seed_seed=301 + seed_offset)
    spec, qt, sd = synth.ik_workload(cfg, batch)
    g = pk.Robot.from_spec(spec)
    ee = g.n_joints - 1
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    targets = pk.pk_fk(g, dev(qt))[:, ee:ee + 1].contiguous()
    return g, ee, targets, dev(sd)


def _compare(a, b):
    q, err, iters, status = [x.cpu().numpy() for x in a]
    q2, err2, iters2, status2 = [x.cpu().numpy() for x in b]
    np.testing.assert_array_equal(status, status2)
    np.testing.assert_array_equal(iters, iters2)
    np.testing.assert_allclose(q, q2, atol=1e-5, rtol=0)
    np.testing.assert_allclose(err, err2, atol=1e-5, rtol=0)


def test_noalloc_matches_workspace_solve_twice():
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    for batch, off in ((2048, 0), (1500, 7)):  # two calls in a row, different sizes and inputs
        g, ee, targets, seeds = _inputs(batch, off)
        ws = torch.empty(pk.pk_ik_workspace_bytes(g, batch, 8), dtype=torch.uint8, device="cuda")
        ref = pk.pk_ik_solve(g, p, [ee], None, targets, seeds, ws)
        got = pk.pk_ik_solve_noalloc(g, p, [ee], None, targets, seeds)
        torch.cuda.synchronize()
        _compare(ref, got)
        assert (got[3] == pk.PK_P_CONVERGED).float().mean().item() > 0.8


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    g, ee, targets, seeds = _inputs(8)
    p = pk.pk_ik_params_default()
    big = 200_000  # 1.6 M seeds of a 7-DoF chain need ~77 MB of scratch
    assert pk.pk_ik_workspace_bytes(g, big, 8) > 32 << 20
    B = big
    t = torch.zeros(B, 1, 12, device="cuda")
    s = torch.zeros(B, 8, 7, device="cuda")
    with pytest.raises(pk.PkError) as e:
        pk.pk_ik_solve_noalloc(g, p, [ee], None, t, s)
    assert e.value.status == pk.PK_ERR_INVALID_ARG
    assert "static scratch" in pk.pk_last_error()


def _tree_inputs(batch, seed_offset=0):
    spec, tips = synth.hand_robot(102)
    g = pk.Robot.from_spec(spec)
    qt = synth.uniform_q(640 + seed_offset, batch, spec.dof_lower, spec.dof_upper)
    sd = synth.uniform_q(650 + seed_offset, (batch, 4), spec.dof_lower, spec.dof_upper)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    targets = pk.pk_fk(g, dev(qt))[:, list(tips)].contiguous()
    kinds = [pk.PK_TARGET_POSITION] * len(tips)
    return g, list(tips), kinds, targets, dev(sd)


def test_noalloc_tree_robot_twice():
    """The warp-per-problem tree kernel (24-DoF hand, five fingertip position
    targets) has a larger per-seed record than the chain kernel; two calls in
    a row through the shared array equal pk_ik_solve with a caller workspace."""
    p = pk.pk_ik_params_default(max_iters=30, early_exit=1, cancel_siblings=0)
    for batch, off in ((700, 0), (333, 3)):
        g, tips, kinds, targets, seeds = _tree_inputs(batch, off)
        ws = torch.empty(pk.pk_ik_workspace_bytes(g, batch, 4), dtype=torch.uint8, device="cuda")
        ref = pk.pk_ik_solve(g, p, tips, kinds, targets, seeds, ws)
        got = pk.pk_ik_solve_noalloc(g, p, tips, kinds, targets, seeds)
        torch.cuda.synchronize()
        _compare(ref, got)


def test_noalloc_sibling_cancellation_flags_start_clear():
    """With sibling cancellation the per-target flags live in the shared
    array: a flag left set by the previous call would stop that target's
    seeds.  A target is solved iff one of its seeds converges, whichever
    seeds were cancelled, so the solved set of each call must equal
    pk_ik_solve's, and every converged answer must meet the tolerances."""
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=1)
    for batch, off in ((3000, 11), (3000, 12)):
        g, ee, targets, seeds = _inputs(batch, off)
        ws = torch.empty(pk.pk_ik_workspace_bytes(g, batch, 8), dtype=torch.uint8, device="cuda")
        ref = pk.pk_ik_solve(g, p, [ee], None, targets, seeds, ws)
        got = pk.pk_ik_solve_noalloc(g, p, [ee], None, targets, seeds)
        torch.cuda.synchronize()
        s_ref, s_got = ref[3].cpu().numpy(), got[3].cpu().numpy()
        np.testing.assert_array_equal(s_got == pk.PK_P_CONVERGED, s_ref == pk.PK_P_CONVERGED)
        err = got[1].cpu().numpy()[s_got == pk.PK_P_CONVERGED]
        assert np.all(err[:, 0] <= p.tol_pos) and np.all(err[:, 1] <= p.tol_rot)


def test_noalloc_empty_batch_and_argument_errors_come_first():
    g, ee, targets, seeds = _inputs(8)
    p = pk.pk_ik_params_default()
    t0, s0 = torch.zeros(0, 1, 12, device="cuda"), torch.zeros(0, 8, 7, device="cuda")
    q, err, iters, status = pk.pk_ik_solve_noalloc(g, p, [ee], None, t0, s0)
    assert q.shape == (0, 7)
    # an unsupported target frame beside an oversized batch reports the target
    big = 200_000
    t = torch.zeros(big, 1, 12, device="cuda")
    s = torch.zeros(big, 8, 7, device="cuda")
    with pytest.raises(pk.PkError):
        pk.pk_ik_solve_noalloc(g, p, [g.n_joints + 5], None, t, s)
    assert "static scratch" not in pk.pk_last_error()
