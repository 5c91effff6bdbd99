"""Trajectory-optimisation extensions of the oracle: the velocity-limit hinge
(Sec. III-C, dt = 1) and swept-sphere collision between consecutive timesteps
(Sec. IV-A).  Pinned by recomputing the rows in numpy from the oracle's FK
frames -- the capsule distance by a dense brute-force search along the segment
instead of the closed-form closest point --, by central differences of the
new rows, and by the normal matrix's block structure (still pentadiagonal:
both row kinds couple neighbouring timesteps only)."""
import numpy as np

import oracle
from paper_2505_03728_gb300 import synth

T, N, S = 6, 7, 4


def f_eta(d, eta):
    return np.where(d <= 0, -d + 0.5 * eta, np.where(d < eta, 0.5 / eta * (eta - d) ** 2, 0.0))


def setup(seed=0, spread=0.35):
    spec = synth.chain_robot(100, 7)
    rb = oracle.Robot.from_dict(spec)
    rng = np.random.default_rng(seed)
    qs = synth.uniform_q(seed + 1, 1, rb.dof_lower, rb.dof_upper)[0]
    x = qs + np.cumsum(rng.normal(0, spread, (T, N)), axis=0)  # fast moves: velocity hinges active
    Tf = oracle.fk(rb, x[T // 2])
    obs = [[*(Tf[j].reshape(3, 4)[:, 3] + rng.normal(0, 0.05, 3)), 0.1] for j in (2, 4, 6)]
    radii = synth.link_spheres(3, 7)
    scene = oracle.Scene(radii, np.array(obs), [0, 0, 1, -5.0])
    goal = oracle.fk(rb, qs)[-1]
    return rb, scene, x, qs, goal, radii, np.array(obs)


def sphere_centres(rb, q):
    Tf = oracle.fk(rb, q).reshape(-1, 3, 4)
    joints = [j for j in range(rb.n_joints) if rb.type[j] != 0] + [rb.n_joints - 1]
    c = []
    for l in range(N):
        pa, pb = Tf[joints[l]][:, 3], Tf[joints[l + 1]][:, 3]
        c.append([pa + (s + 0.5) / S * (pb - pa) for s in range(S)])
    return np.array(c)  # [N][S][3]


def rows(rb, prm, scene, x, qs, goal):
    r, J = oracle.traj_residual(rb, prm, scene, x, qs, goal)
    n_vel, n_sw, n_5 = (T - 1) * N, (T - 1) * N * S * 3, 2 * N * max(T - 4, 0)  # five-point rows come last
    end = len(r) - n_5
    return r, J, slice(end - n_sw - n_vel, end - n_sw), slice(end - n_sw, end)


def test_rows_recomputed_in_numpy():
    rb, scene, x, qs, goal, radii, obs = setup()
    prm = oracle.TrajParams(w_vlimit=3.0, v_max=0.2, w_swept=7.0, eta=0.03)
    r, J, vel, sw = rows(rb, prm, scene, x, qs, goal)
    dv = np.abs(np.diff(x, axis=0)) - 0.2
    np.testing.assert_allclose(r[vel], 3.0 * np.maximum(dv, 0).ravel(), atol=1e-12)
    assert np.count_nonzero(r[vel]) > 5
    want = []
    us = np.linspace(0, 1, 200001)
    for t in range(T - 1):
        c0, c1 = sphere_centres(rb, x[t]), sphere_centres(rb, x[t + 1])
        for l in range(N):
            for s in range(S):
                seg = c0[l, s] + us[:, None] * (c1[l, s] - c0[l, s])
                for o in obs:
                    dist = np.sqrt(((seg - o[:3]) ** 2).sum(axis=1)).min()
                    want.append(dist - radii[l, s] - o[3])
    np.testing.assert_allclose(r[sw], 7.0 * f_eta(np.array(want), 0.03), atol=2e-6)
    assert np.count_nonzero(r[sw]) > 5


def test_new_rows_jacobian_matches_central_differences():
    rb, scene, x, qs, goal, radii, obs = setup(seed=3)
    prm = oracle.TrajParams(w_vlimit=3.0, v_max=0.2, w_swept=7.0, eta=0.03)
    r, J, vel, sw = rows(rb, prm, scene, x, qs, goal)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for a in range(x.size):
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[a] += h
        xm[a] -= h
        Jfd[:, a] = (oracle.traj_residual(rb, prm, scene, xp.reshape(x.shape), qs, goal, False)
                     - oracle.traj_residual(rb, prm, scene, xm.reshape(x.shape), qs, goal, False)) / (2 * h)
    dv = (np.abs(np.diff(x, axis=0)) - 0.2).ravel()
    smooth_v = np.abs(dv) > 1e-4
    idx_v = np.arange(vel.start, vel.stop)[smooth_v]
    np.testing.assert_allclose(J[idx_v], Jfd[idx_v], atol=1e-6)
    f = r[sw] / 7.0
    kink = (np.abs(f - 0.5 * 0.03) < 1e-4) | ((f > 0) & (f < 1e-7))
    idx_s = np.arange(sw.start, sw.stop)[~kink]
    err = np.abs(J[idx_s] - Jfd[idx_s]) / np.maximum(1.0, np.abs(J[idx_s]))
    assert err.max() <= 1e-5, err.max()


def test_normal_matrix_stays_block_pentadiagonal_and_banded_equals_dense():
    rb, scene, x, qs, goal, radii, obs = setup(seed=5)
    prm = oracle.TrajParams(w_vlimit=3.0, v_max=0.2, w_swept=7.0, eta=0.03)
    f, A, g = oracle.traj_normal(rb, prm, scene, x, qs, goal)
    for t in range(T):
        for u in range(T):
            if abs(t - u) > 2:
                assert np.all(A[t * N:(t + 1) * N, u * N:(u + 1) * N] == 0.0)
    A2 = A + 1e-2 * np.eye(A.shape[0])
    np.testing.assert_allclose(oracle.banded_cholesky(A2, T, N), np.linalg.cholesky(A2), rtol=1e-10, atol=1e-12)
    a = oracle.traj_solve(rb, oracle.TrajParams(iters=6, banded=1, w_vlimit=3.0, v_max=0.2, w_swept=7.0, eta=0.03),
                          scene, x[None], qs[None], goal[None])
    b = oracle.traj_solve(rb, oracle.TrajParams(iters=6, banded=0, w_vlimit=3.0, v_max=0.2, w_swept=7.0, eta=0.03),
                          scene, x[None], qs[None], goal[None])
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-9)


def test_five_point_rows_are_the_stencils_and_widen_the_band_to_four():
    rb, scene, x, qs, goal, radii, obs = setup(seed=7)
    Tl = 9
    rng = np.random.default_rng(7)
    x = qs + np.cumsum(rng.normal(0, 0.1, (Tl, N)), axis=0)
    prm = oracle.TrajParams(w_acc5=2.0, w_jerk=3.0)
    r, J = oracle.traj_residual(rb, prm, scene, x, qs, goal)
    nr = N * (Tl - 4)
    acc = (-x[4:] + 16 * x[3:-1] - 30 * x[2:-2] + 16 * x[1:-3] - x[:-4]) / 12
    jerk = (x[4:] - 2 * x[3:-1] + 2 * x[1:-3] - x[:-4]) / 2
    np.testing.assert_allclose(r[-2 * nr:-nr], 2.0 * acc.ravel(), atol=1e-12)
    np.testing.assert_allclose(r[-nr:], 3.0 * jerk.ravel(), atol=1e-12)
    # a quadratic trajectory has zero jerk and constant acceleration (exact stencils)
    tt = np.arange(Tl, dtype=float)[:, None]
    xq = qs + 0.01 * tt + 0.003 * tt ** 2
    rq, _ = oracle.traj_residual(rb, prm, scene, xq, qs, goal)
    np.testing.assert_allclose(rq[-nr:], 0.0, atol=1e-12)
    np.testing.assert_allclose(rq[-2 * nr:-nr], 2.0 * 0.006, atol=1e-12)
    # closed forms: the fourth-order acceleration stencil is exact up to degree 5,
    # the second-order jerk stencil up to degree 4 (dt = 1): rows equal the
    # analytic derivatives of a quintic / quartic at the interior steps
    cq = rng.normal(0, 1e-3, (6, N))  # x(t) = sum_k c_k t^k
    xp = qs + sum(cq[k] * tt ** k for k in range(1, 6))
    rp, _ = oracle.traj_residual(rb, prm, scene, xp, qs, goal)
    ti = tt[2:-2]
    d2 = sum(k * (k - 1) * cq[k] * ti ** (k - 2) for k in range(2, 6))
    np.testing.assert_allclose(rp[-2 * nr:-nr], 2.0 * d2.ravel(), rtol=1e-9, atol=1e-12)
    xp4 = qs + sum(cq[k] * tt ** k for k in range(1, 5))
    rp4, _ = oracle.traj_residual(rb, prm, scene, xp4, qs, goal)
    d3 = sum(k * (k - 1) * (k - 2) * cq[k] * ti ** (k - 3) for k in range(3, 5))
    np.testing.assert_allclose(rp4[-nr:], 3.0 * d3.ravel(), rtol=1e-9, atol=1e-12)
    f, A, g = oracle.traj_normal(rb, prm, scene, x, qs, goal)
    nz = lambda t, u: np.any(A[t * N:(t + 1) * N, u * N:(u + 1) * N] != 0.0)
    assert nz(6, 2) and not nz(7, 2)  # blocks at distance 4 are filled, beyond 4 empty
    A2 = A + 1e-2 * np.eye(A.shape[0])
    np.testing.assert_allclose(oracle.banded_cholesky(A2, Tl, N, band=4), np.linalg.cholesky(A2), rtol=1e-10,
                               atol=1e-12)
    a = oracle.traj_solve(rb, oracle.TrajParams(iters=6, banded=1, w_acc5=2.0, w_jerk=3.0), scene, x[None],
                          qs[None], goal[None])
    b = oracle.traj_solve(rb, oracle.TrajParams(iters=6, banded=0, w_acc5=2.0, w_jerk=3.0), scene, x[None],
                          qs[None], goal[None])
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-9)
