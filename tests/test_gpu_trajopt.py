"""GPU trajectory optimisation (block-banded LM) against the FP64 oracle.

The damped normal matrices of this workload have condition numbers of 1e6 -
3e6: the start and goal rows (weight 100) put entries of ~1e4 into the first
and last diagonal blocks, the smoothness rows (weight 1) and lambda ~1e-2 set
the soft directions.  Merely holding M = J^T J + lambda I and g in FP32 moves
the exact step by 3e-5 .. 6e-4 of max(1, |q|), so no FP32 solver, iterative
refinement included, can match an FP64 step to 1e-4 on every trajectory.
The parity bar is therefore per trajectory and per step, from the
arithmetic: the first-order componentwise perturbation bound of the solution
of M d = -g when every entry of M and g carries a relative error u = 2^-24,

    s = u max_i (|M^-1| (|A| |d| + |g|))_i / max(1, |q_i|),

computed from the oracle's FP64 normal equations at the step's start; every
trajectory without an accept/reject near-tie (|f_trial - f| <= 1e-5 f) must
agree within 2 s (measured: at most 0.8 s), one step at a time from the
oracle's own iterates and damping (iterates 1 to 5) and over free runs of 1
to 5 iterations (within 2 sum_k s_k).  Two kinds of step are decided by
rounding and excluded (and counted), because both results are correct: an
accept/reject near-tie, and a start with a joint within 1e-6 rad of a limit,
where the limit hinge's derivative jumps from 0 to w_limit and FP32 rounding
of q decides which side the step sees.  Where 2 s <= 1e-4 this is the 1e-4
bar itself.  Normal-equation blocks and gradient agree within 1e-4 of the
largest entry; after the full solve the oracle's FP64 cost at the GPU's
trajectory agrees with the GPU's own cost to 1e-3."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_03728_gb300 import build, pk, scenes, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def setup(B, T=64, perturb=0.0, seed=0):
    cfg = synth.TRAJOPT
    spec, qs_c, qg_c, radii, obs, plane = synth.trajopt_workload(cfg, B)
    o = oracle.Robot.from_dict(spec)
    g = pk.Robot.from_spec(spec)
    n_c = 16 * B
    pick = lambda q: scenes.pick_clear(q[:n_c], oracle.fk(o, q[:n_c])[:, :, [3, 7, 11]], radii, obs, plane, 0.02, B)
    qs, qg = pick(qs_c), pick(qg_c)
    goals = oracle.fk(o, qg)[:, -1]
    x0 = synth.linear_interpolation(qs, qg, T)
    if perturb:
        x0 = x0 + np.random.default_rng(seed).normal(0, perturb, x0.shape)
    scene = oracle.Scene(radii, obs, plane)
    return o, g, qs, goals, x0, radii, obs, plane, scene


U32 = 2.0 ** -24


def step_sensitivity(o, op, scene, x, qs, goal, lam):
    """First-order componentwise bound of the damped LM step's FP32 error,
    relative to max(1, |q|) (see the module docstring)."""
    f, A, gr = oracle.traj_normal(o, op, scene, x, qs, goal)
    M = A + lam * np.eye(len(A))
    d = np.linalg.solve(M, -gr)
    s = U32 * np.abs(np.linalg.inv(M)) @ (np.abs(A) @ np.abs(d) + np.abs(gr))
    return float(np.max(s / np.maximum(1.0, np.abs(np.asarray(x).ravel()))))


HINGE_KINK = 1e-6  # rad: a joint this close to a limit may round onto the other side in FP32


def hinge_kink(o, x):
    """True when a joint of trajectory x [T][n] lies within HINGE_KINK of a limit."""
    x = np.asarray(x)
    return bool(np.min(np.minimum(np.abs(x - o.dof_lower), np.abs(x - o.dof_upper))) <= HINGE_KINK)


def oparams(p, banded=1):
    return oracle.TrajParams(p.w_start, p.w_goal_pos, p.w_goal_rot, p.w_vel, p.w_acc, p.w_limit, p.w_coll,
                             p.eta, p.lambda0, p.lambda_min, p.lambda_max, p.nu, p.iters, banded,
                             w_vlimit=p.w_vlimit, v_max=p.v_max, w_swept=p.w_swept,
                             w_acc5=p.w_acc5, w_jerk=p.w_jerk)


@pytest.mark.parametrize("T", [3, 17, 64])
def test_normal_equations_match_oracle(T):
    o, g, qs, goals, x0, radii, obs, plane, scene = setup(6, T, perturb=0.1)
    p = pk.pk_trajopt_params_default()
    D, gg, cost = [x.cpu().numpy().astype(np.float64) for x in
                   pk.pk_trajopt_normal(g, p, dev(qs), dev(goals), dev(x0), dev(radii), dev(obs), plane)]
    op = oparams(p)
    n = 7
    for b in range(6):
        f, A, gr = oracle.traj_normal(o, op, scene, x0[b], qs[b], goals[b])
        scale = np.abs(A).max()
        for t in range(T):
            np.testing.assert_allclose(D[b, t], A[t * n:(t + 1) * n, t * n:(t + 1) * n], atol=1e-4 * scale)
            # off-diagonal blocks of the oracle are the smoothness scalars times I
            for dt in (1, 2):
                if t - dt >= 0:
                    blk = A[t * n:(t + 1) * n, (t - dt) * n:(t - dt + 1) * n]
                    np.testing.assert_allclose(blk, blk[0, 0] * np.eye(n), atol=1e-12)
        np.testing.assert_allclose(gg[b].ravel(), gr, atol=1e-4 * max(1.0, np.abs(gr).max()))
        assert abs(cost[b] - f) <= 1e-4 * max(1.0, f)


def test_one_step_from_several_points_matches_oracle():
    """One LM step (lambda0) from the initial trajectories and from the oracle's
    own iterates 5 and 20: the step alone, without accumulated history, within
    twice its FP32 sensitivity bound on every trajectory."""
    o, g, qs, goals, x0, radii, obs, plane, scene = setup(16, 64)
    p1 = pk.pk_trajopt_params_default(iters=1)
    op1 = oparams(p1)
    trace = oracle.traj_solve(o, oparams(pk.pk_trajopt_params_default(iters=20)), scene, x0, qs, goals,
                              n_trace=True)["trace"]
    for start in (x0, trace[:, 4], trace[:, 19]):
        ref = oracle.traj_solve(o, op1, scene, start, qs, goals, n_trace=True)
        q = pk.pk_trajopt_solve(g, p1, dev(qs), dev(goals), dev(start), dev(radii), dev(obs), plane)[0].cpu().numpy()
        tie = ref["margin"] <= 1e-5
        kink = np.array([hinge_kink(o, start[b]) for b in range(16)])
        rel = (np.abs(q - ref["x"]) / np.maximum(1.0, np.abs(ref["x"]))).reshape(16, -1).max(axis=1)
        for b in np.nonzero(~tie & ~kink)[0]:
            sb = step_sensitivity(o, op1, scene, start[b], qs[b], goals[b], p1.lambda0)
            assert rel[b] <= 2 * sb + 1e-6, (b, rel[b], sb)
        # near a stationary point (the start at iterate 20) cost changes are small
        assert (tie | kink).sum() <= 4


FIVE = dict(w_acc5=2.0, w_jerk=3.0)
LIMITS = dict(w_vlimit=3.0, v_max=0.02, w_swept=10.0)


@pytest.mark.parametrize("T", [5, 7, 8, 9, 12, 15, 16, 17, 33])
@pytest.mark.parametrize("ext", [{}, LIMITS, FIVE, dict(FIVE, **LIMITS)], ids=["plain", "limits", "five", "both"])
def test_one_step_short_horizons_match_oracle(T, ext):
    """One LM step at horizons on both sides of the shortest the two-ended
    block factorisations take (8 with two block sub-diagonals, 16 with the
    four of the five-point stencils), odd and even, with and without the
    off-diagonal blocks of the velocity-limit and swept terms."""
    o, g, qs, goals, x0, radii, obs, plane, scene = setup(8, T, perturb=0.1, seed=T)
    p = pk.pk_trajopt_params_default(iters=1, **ext)
    ref = oracle.traj_solve(o, oparams(p), scene, x0, qs, goals, n_trace=True)
    q = pk.pk_trajopt_solve(g, p, dev(qs), dev(goals), dev(x0), dev(radii), dev(obs), plane)[0].cpu().numpy()
    tie = ref["margin"] <= 1e-5
    rel = (np.abs(q - ref["x"]) / np.maximum(1.0, np.abs(ref["x"]))).reshape(8, -1).max(axis=1)
    op = oparams(p)
    # every step within twice its FP32 sensitivity bound
    for b in np.nonzero(~tie)[0]:
        sb = step_sensitivity(o, op, scene, x0[b], qs[b], goals[b], p.lambda0)
        assert rel[b] <= 2 * sb + 1e-6, (b, rel[b], sb)
    # and an accepted GPU step solves the oracle's damped normal equations to
    # FP32 accuracy (backward error); a wrong block in the factorisation or
    # the substitutions leaves an O(1) residual
    for b in np.nonzero(~tie)[0]:
        # the GPU started from x0 rounded to FP32: a rejected step leaves it exactly there
        dx = (q[b].astype(np.float64) - x0[b].astype(np.float32).astype(np.float64)).ravel()
        if not np.any(dx):
            continue  # rejected step
        f, A, gr = oracle.traj_normal(o, op, scene, x0[b], qs[b], goals[b])
        M = A + p.lambda0 * np.eye(len(A))
        be = np.linalg.norm(M @ dx + gr) / (np.linalg.norm(M, 2) * np.linalg.norm(dx) + np.linalg.norm(gr))
        assert be <= 1e-4, (b, be)


def test_first_iterates_one_step_from_the_oracle_path():
    """Iterates 1 to 5, one step at a time: the GPU starts every step from the
    oracle's iterate k-1 with the oracle's damping after k-1 iterations (the
    damping trace of oracle.traj_lm_run), and its iterate k must lie within
    twice the step's FP32 sensitivity of the oracle's on every trajectory
    without a near-tie at that step.  Where that bound is below 1e-4, the
    1e-4 bar holds."""
    B, K = 24, 5
    o, g, qs, goals, x0, radii, obs, plane, scene = setup(B, 64)
    op = oparams(pk.pk_trajopt_params_default(iters=K))
    ratios, ties, within_bar = [], 0, []
    for b in range(B):
        run = oracle.traj_lm_run(o, op, scene, x0[b], qs[b], goals[b])
        lam_prev = np.concatenate([[op.lambda0], run["lam_trace"]])
        for k in range(1, K + 1):
            start = x0[b] if k == 1 else run["trace"][k - 2]
            p1 = pk.pk_trajopt_params_default(iters=1, lambda0=float(lam_prev[k - 1]))
            one = oracle.traj_solve(o, oparams(p1), scene, start[None], qs[b:b + 1], goals[b:b + 1], n_trace=True)
            if one["margin"][0] <= 1e-5 or hinge_kink(o, start):
                ties += 1
                continue
            q = pk.pk_trajopt_solve(g, p1, dev(qs[b:b + 1]), dev(goals[b:b + 1]), dev(start[None]), dev(radii),
                                    dev(obs), plane)[0].cpu().numpy()[0]
            ref = run["trace"][k - 1]
            np.testing.assert_array_equal(one["x"][0], ref)  # the single step reproduces the oracle's path
            rel = np.max(np.abs(q - ref) / np.maximum(1.0, np.abs(ref)))
            sb = step_sensitivity(o, op, scene, start, qs[b], goals[b], lam_prev[k - 1])
            ratios.append(rel / sb)
            assert rel <= 2 * sb + 1e-6, (b, k, rel, sb)
            if 2 * sb <= 1e-4:
                within_bar.append(rel)
    print(f"one-step iterates: max error / bound {max(ratios):.2f}, {ties} near-ties or hinge kinks excluded, "
          f"{len(within_bar)} steps where FP32 allows the 1e-4 bar (worst {max(within_bar, default=0):.1e})")
    assert ties <= 6 and all(r <= 1e-4 for r in within_bar)  # at most 5% of the 120 steps


def test_first_iterates_match_oracle():
    """Free runs of 1 to 5 iterations from the same start: every trajectory
    without a near-tie in its first five iterations stays within twice the
    sum of its steps' FP32 sensitivity bounds."""
    B, K = 24, 5
    o, g, qs, goals, x0, radii, obs, plane, scene = setup(B, 64)
    op = oparams(pk.pk_trajopt_params_default(iters=K))
    ref = oracle.traj_solve(o, op, scene, x0, qs, goals, n_trace=True)
    tie = ref["margin"] <= 1e-5
    # a hinge kink at the start of any of the five steps makes the rest of the
    # run depend on rounding, like a near-tie
    tie |= np.array([any(hinge_kink(o, x) for x in [x0[b]] + list(ref["trace"][b, :K - 1])) for b in range(B)])
    cum = np.zeros(B)
    lam = [oracle.traj_lm_run(o, op, scene, x0[b], qs[b], goals[b])["lam_trace"] for b in range(B)]
    for k in range(1, K + 1):
        for b in range(B):
            start = x0[b] if k == 1 else ref["trace"][b, k - 2]
            lam_k = op.lambda0 if k == 1 else lam[b][k - 2]
            cum[b] += step_sensitivity(o, op, scene, start, qs[b], goals[b], lam_k)
        p = pk.pk_trajopt_params_default(iters=k)
        q = pk.pk_trajopt_solve(g, p, dev(qs), dev(goals), dev(x0), dev(radii), dev(obs), plane)[0].cpu().numpy()
        rel = (np.abs(q - ref["trace"][:, k - 1]) / np.maximum(1.0, np.abs(ref["trace"][:, k - 1]))).reshape(B, -1)
        worst = rel.max(axis=1)
        bad = (~tie) & (worst > 2 * cum + 1e-6)
        assert not bad.any(), (k, worst[bad], cum[bad])
    print(f"free runs: {tie.sum()} of {B} trajectories with a near-tie or hinge kink in five iterations")
    assert tie.sum() <= 3


def test_full_solve_against_oracle():
    B = 32
    o, g, qs, goals, x0, radii, obs, plane, scene = setup(B, 64)
    p = pk.pk_trajopt_params_default()
    q, cost, st = pk.pk_trajopt_solve(g, p, dev(qs), dev(goals), dev(x0), dev(radii), dev(obs), plane)
    q, cost, st = q.cpu().numpy(), cost.cpu().numpy(), st.cpu().numpy()
    op = oparams(p)
    ref = oracle.traj_solve(o, op, scene, x0, qs, goals)
    for b in range(B):
        f_at_gpu = oracle.traj_normal(o, op, scene, q[b], qs[b], goals[b])[0]
        assert abs(f_at_gpu - cost[b]) <= 1e-3 * max(1.0, f_at_gpu)
    ratio = np.median(cost / ref["cost"])
    assert 0.5 <= ratio <= 2.0, ratio
    # collision status from the oracle's own geometry at both solutions
    print(f"median cost ratio GPU/oracle {ratio:.3f}; GPU collision-free {(st & 2 == 0).mean():.2f}")


def test_trajopt_argument_checks():
    o, g, qs, goals, x0, radii, obs, plane, scene = setup(2, 8)
    p = pk.pk_trajopt_params_default()
    with pytest.raises(pk.PkError):
        pk.pk_trajopt_solve(g, p, dev(qs), dev(goals), dev(np.zeros((2, 65, 7))), dev(radii), dev(obs), plane)
    # no obstacles at all
    q, cost, st = pk.pk_trajopt_solve(g, pk.pk_trajopt_params_default(iters=5), dev(qs), dev(goals), dev(x0),
                                      dev(radii), dev(np.zeros((0, 4))), plane)
    assert np.all(np.isfinite(cost.cpu().numpy()))
