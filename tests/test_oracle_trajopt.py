"""Pins for the FP64 trajectory-optimisation oracle: the Eq. 1 activation by
hand-computed values and its C1 continuity, the full residual Jacobian by
central differences, the normal matrix against J^T J (numpy) and its block
pentadiagonal structure, the block-banded Cholesky against LAPACK, and LM on
special cases whose minimisers are known in closed form."""
import numpy as np
import pytest

import oracle
from paper_2505_03728_gb300 import synth


def test_activation_hand_values_and_c1():
    eta = 0.02
    for d, f in [(-0.01, 0.02), (0.0, 0.01), (0.005, 0.5 / 0.02 * 0.015 ** 2), (0.02, 0.0), (0.05, 0.0)]:
        assert abs(oracle.coll_activation(d, eta)[0] - f) < 1e-15
    for x in (0.0, eta):
        fl, dl = oracle.coll_activation(x - 1e-9, eta)
        fr, dr = oracle.coll_activation(x + 1e-9, eta)
        assert abs(fl - fr) < 1e-8 and abs(dl - dr) < 1e-6


def _small(T=5, seed=0, n_obs=3):
    spec = synth.chain_robot(100, 7)
    rb = oracle.Robot.from_dict(spec)
    rng = np.random.default_rng(seed)
    qs = synth.uniform_q(seed + 1, 1, rb.dof_lower, rb.dof_upper)[0]
    qg = synth.uniform_q(seed + 2, 1, rb.dof_lower, rb.dof_upper)[0]
    x = synth.linear_interpolation(qs[None], qg[None], T)[0] + rng.normal(0, 0.05, (T, 7))
    # obstacles placed on the arm so that collision rows are active
    Tf = oracle.fk(rb, x[T // 2])
    obs = []
    for j in (2, 4, 6)[:n_obs]:
        c = Tf[j].reshape(3, 4)[:, 3] + rng.normal(0, 0.05, 3)
        obs.append([*c, 0.1])
    radii = synth.link_spheres(3, 7)
    scene = oracle.Scene(radii, np.array(obs), [0, 0, 1, -0.15])
    goal = oracle.fk(rb, qg)[-1]
    return rb, scene, x, qs, goal


def test_residual_jacobian_matches_central_fd():
    rb, scene, x, qs, goal = _small()
    prm = oracle.TrajParams()
    r, J = oracle.traj_residual(rb, prm, scene, x, qs, goal)
    # velocity-limit, swept-sphere and five-point rows (off here) follow the collision rows
    ext = 4 * 7 + 4 * 7 * 4 * 3 + 2 * 7 * 1
    coll = slice(len(r) - ext - 5 * 7 * 4 * 4, len(r) - ext)
    assert np.count_nonzero(r[coll]) > 5  # some collision rows active
    assert np.count_nonzero(r[len(r) - ext:]) == 0
    h = 1e-6
    Jfd = np.zeros_like(J)
    for a in range(x.size):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[a] += h
        xm[a] -= h
        Jfd[:, a] = (oracle.traj_residual(rb, prm, scene, xp.reshape(x.shape), qs, goal, False)
                     - oracle.traj_residual(rb, prm, scene, xm.reshape(x.shape), qs, goal, False)) / (2 * h)
    # rows next to an activation kink (d = 0 or d = eta) are not differentiable at FD scale
    f = r / prm.w_coll
    near_kink = np.zeros(len(r), bool)
    fc = f[coll]
    near_kink[coll] = (np.abs(fc - 0.5 * prm.eta) < 1e-4) | ((fc > 0) & (fc < 1e-7))
    err = np.abs(J - Jfd) / np.maximum(1.0, np.abs(J))
    assert err[~near_kink].max() <= 1e-6


def test_normal_matrix_is_jtj_and_block_pentadiagonal():
    rb, scene, x, qs, goal = _small(T=8, seed=1)
    prm = oracle.TrajParams()
    f, A, g = oracle.traj_normal(rb, prm, scene, x, qs, goal)
    r, J = oracle.traj_residual(rb, prm, scene, x, qs, goal)
    np.testing.assert_allclose(A, J.T @ J, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(g, J.T @ r, rtol=1e-12, atol=1e-10)
    assert abs(f - 0.5 * r @ r) <= 1e-12 * max(1, f)
    n = 7
    for t in range(8):
        for u in range(8):
            if abs(t - u) > 2:
                assert np.all(A[t * n:(t + 1) * n, u * n:(u + 1) * n] == 0.0)


def test_banded_cholesky_matches_lapack():
    rb, scene, x, qs, goal = _small(T=10, seed=2)
    _, A, _ = oracle.traj_normal(rb, oracle.TrajParams(), scene, x, qs, goal)
    A = A + 1e-2 * np.eye(A.shape[0])
    L = oracle.banded_cholesky(A, 10, 7)
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-10, atol=1e-12)
    assert oracle.banded_cholesky(-np.eye(70), 10, 7) is None


def test_banded_and_dense_solves_agree():
    rb, scene, x, qs, goal = _small(T=6, seed=3)
    goals = goal[None]
    a = oracle.traj_solve(rb, oracle.TrajParams(iters=8, banded=1), scene, x[None], qs[None], goals)
    b = oracle.traj_solve(rb, oracle.TrajParams(iters=8, banded=0), scene, x[None], qs[None], goals)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-9)


def test_lm_costs_decrease():
    rb, scene, x, qs, goal = _small(T=6, seed=4)
    out = oracle.traj_solve(rb, oracle.TrajParams(iters=20), scene, x[None], qs[None], goal[None], n_trace=True)
    prm = oracle.TrajParams()
    costs = [oracle.traj_normal(rb, prm, scene, x, qs, goal)[0]]
    for k in range(20):
        costs.append(oracle.traj_normal(rb, prm, scene, out["trace"][0, k], qs, goal)[0])
    assert all(b <= a for a, b in zip(costs, costs[1:]))
    assert costs[-1] < 0.5 * costs[0]


def test_closed_form_minimisers():
    """Start + velocity only: the minimiser is constant at q_start.  Start +
    acceleration only: every minimiser is a straight line in t."""
    spec = synth.chain_robot(100, 7)
    rb = oracle.Robot.from_dict(spec)
    scene = oracle.Scene(np.full((7, 4), 0.01), np.zeros((0, 4)), [0, 0, 1, -100.0])
    rng = np.random.default_rng(5)
    T = 8
    qs = rng.uniform(-1, 1, 7)
    x0 = rng.uniform(-1, 1, (T, 7))
    goal = synth.EYE12
    p = oracle.TrajParams(w_goal_pos=0, w_goal_rot=0, w_acc=0, w_limit=0, w_coll=0, iters=60)
    out = oracle.traj_solve(rb, p, scene, x0[None], qs[None], goal[None])
    np.testing.assert_allclose(out["x"][0], np.tile(qs, (T, 1)), atol=1e-8)
    p = oracle.TrajParams(w_goal_pos=0, w_goal_rot=0, w_vel=0, w_limit=0, w_coll=0, iters=200)
    out = oracle.traj_solve(rb, p, scene, x0[None], qs[None], goal[None])
    x = out["x"][0]
    np.testing.assert_allclose(x[0], qs, atol=1e-8)
    np.testing.assert_allclose(x[2:] - 2 * x[1:-1] + x[:-2], 0, atol=1e-6)
