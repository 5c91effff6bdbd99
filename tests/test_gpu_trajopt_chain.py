"""The trajectory workload as Sec. IV-A sets it up: the goal configuration comes
from IK (multi-start LM from seed-network proposals for the goal pose) and
must be collision-free (pk_ik_select_clear: the lowest-cost converged seed
whose link spheres clear the scene), the initial trajectory is the linear
interpolation from the start configuration to it (pk_trajopt_interpolate),
and the block-banded LM refines that.  Every converged IK answer and every
trajectory that reports its goal reached is re-checked in FP64 with the
oracle's forward kinematics; the selection rule is checked against each
seed solved alone and the oracle's FP64 sphere clearances."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_03728_gb300 import build, pk, scenes, synth
from test_gpu_trajopt import dev, setup

MARGIN = 0.02

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


@pytest.mark.parametrize("T", [1, 2, 3, 17, 64])
def test_interpolate_matches_linear_interpolation(T):
    rng = np.random.default_rng(T)
    q0, q1 = rng.uniform(-2.8, 2.8, (2, 37, 7))
    got = pk.pk_trajopt_interpolate(dev(q0), dev(q1), T).cpu().numpy()
    ref = synth.linear_interpolation(q0.astype(np.float32), q1.astype(np.float32), T)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-6)
    np.testing.assert_array_equal(got[:, 0], q0.astype(np.float32))
    if T > 1:
        np.testing.assert_allclose(got[:, -1], q1.astype(np.float32), rtol=0, atol=1e-6)


def _goal_ik(B, T, n_seeds=8, train=True):
    o, g, qs, goals, x0_gt, radii, obs, plane, scene = setup(B, T)
    ee = o.n_joints - 1
    goals_d = dev(goals).reshape(B, 1, 12).contiguous()
    if train:
        net = pk.SeedNet(g, [ee], K=n_seeds, width=512, depth=4, seed=5)
        pk.pk_seednet_train(net, pk.pk_train_params_default(epochs=2, steps_per_epoch=150, batch=4096))
        seeds = pk.pk_seednet_infer(net, goals_d)
    else:
        seeds = dev(synth.uniform_q(77, (B, n_seeds), o.dof_lower, o.dof_upper))
    p_ik = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    ws = torch.empty(pk.pk_ik_workspace_bytes(g, B, n_seeds), dtype=torch.uint8, device="cuda")
    out = pk.pk_ik_solve(g, p_ik, [ee], None, goals_d, seeds, ws)
    pk.pk_ik_select_clear(g, ws, n_seeds, dev(radii), dev(obs), plane, MARGIN, out=out)
    return o, g, qs, goals, goals_d, radii, obs, plane, seeds, p_ik, out


def test_select_clear_picks_the_clear_converged_seed():
    B, S = 96, 8
    o, g, qs, goals, goals_d, radii, obs, plane, seeds, p_ik, out = _goal_ik(B, 64, S, train=False)
    q, err, iters, st = [x.cpu().numpy() for x in out]
    ee = o.n_joints - 1
    # every seed alone (problems are independent, so each equals its share of the multi-start solve)
    per = [pk.pk_ik_solve(g, p_ik, [ee], None, goals_d, seeds[:, s:s + 1].contiguous()) for s in range(S)]
    qs_ = np.stack([x[0].cpu().numpy() for x in per], 1)
    conv = np.stack([x[3].cpu().numpy() == pk.PK_P_CONVERGED for x in per], 1)
    pts = oracle.fk(o, qs_.reshape(-1, 7).astype(np.float64))[:, :, [3, 7, 11]]
    clear = scenes.clearance(pts, radii, obs, np.asarray(plane, np.float64)).reshape(B, S)
    tg = oracle.Targets([ee])
    prm = oracle.IkParams()
    checked = 0
    for b in range(B):
        if np.any(conv[b] & (np.abs(clear[b] - MARGIN) < 1e-4)):
            continue  # a clearance within FP32 reach of the margin
        cand = conv[b] & (clear[b] > MARGIN)
        pick = np.nonzero(np.all(qs_[b] == q[b], axis=1))[0]
        assert len(pick) >= 1, b  # the answer is one of the seeds' results, bit for bit
        if cand.any():
            assert cand[pick].any(), (b, clear[b], conv[b])
            cost = [0.5 * np.sum(oracle.ik_residual(o, prm, tg, goals[b][None], qs_[b, s], jacobian=False) ** 2)
                    for s in np.nonzero(cand)[0]]
            f_pick = 0.5 * np.sum(oracle.ik_residual(o, prm, tg, goals[b][None], q[b], jacobian=False) ** 2)
            assert f_pick <= min(cost) * (1 + 1e-4) + 1e-12
            checked += 1
        elif conv[b].any():
            assert conv[b][pick].any()
    assert checked >= B // 2


def test_goal_from_seednet_ik_then_trajopt():
    B, T = 64, 64
    o, g, qs, goals, goals_d, radii, obs, plane, seeds, p_ik, out = _goal_ik(B, T)
    ee = o.n_joints - 1
    q_goal, err, iters, st = out
    conv = st.cpu().numpy() == pk.PK_P_CONVERGED
    qg = q_goal.cpu().numpy().astype(np.float64)
    tg = oracle.Targets([ee])
    for b in np.nonzero(conv)[0]:
        pe, re = oracle.ik_errors(o, tg, goals[b][None], qg[b])
        assert pe <= p_ik.tol_pos * 1.01 + 1e-6 and re <= p_ik.tol_rot * 1.01 + 1e-6, (b, pe, re)
    assert conv.mean() >= 0.9
    x0 = pk.pk_trajopt_interpolate(dev(qs), q_goal, T)
    tp = pk.pk_trajopt_params_default()
    q, cost, status = pk.pk_trajopt_solve(g, tp, dev(qs), dev(goals), x0, dev(radii), dev(obs), plane)
    q, status = q.cpu().numpy().astype(np.float64), status.cpu().numpy()
    reached = (status & pk.PK_T_GOAL_MISSED) == 0
    for b in np.nonzero(reached)[0]:
        pe, re = oracle.ik_errors(o, tg, goals[b][None], q[b, -1])
        assert pe <= tp.tol_pos * 1.01 + 1e-6 and re <= tp.tol_rot * 1.01 + 1e-6, (b, pe, re)
    print(f"IK converged {conv.mean():.3f}; goal reached {reached.mean():.3f}; "
          f"collision-free {np.mean((status & pk.PK_T_COLLISION) == 0):.3f}")
    assert reached.mean() >= 0.9
