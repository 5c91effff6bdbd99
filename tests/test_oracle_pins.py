"""Pins for the FP64 CPU oracle (forward kinematics, SE(3) log and Jacobians,
IK residuals, analytic Jacobian, Cholesky, Levenberg-Marquardt).

Every check here compares the oracle with something other than itself: an
independent product-of-exponentials FK written with scipy's matrix
exponential, textbook closed forms (single joint, 2-link planar arm), central
finite differences, LAPACK (numpy.linalg.solve), brute-force grid search, the
power series of the SE(3) left Jacobian, and invariants (orthonormality,
monotone accepted cost).  The paper prints no worked example (Sec. V tables
use the Franka Panda and cuRobo, which are not available), so no printed value
can pin the oracle.
"""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_2505_03728_gb300 import synth


# ---------------------------------------------------------------- helpers
def hat(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]], dtype=float)


def twist_mat(xi):
    M = np.zeros((4, 4))
    M[:3, :3] = hat(xi[3:])
    M[:3, 3] = xi[:3]
    return M


def to44(T12):
    M = np.eye(4)
    M[:3, :] = np.asarray(T12).reshape(3, 4)
    return M


def to12(M):
    return M[:3, :].reshape(12)


def ad(xi):
    A = np.zeros((6, 6))
    A[:3, :3] = hat(xi[3:])
    A[:3, 3:] = hat(xi[:3])
    A[3:, 3:] = hat(xi[3:])
    return A


def random_twist(rng, theta):
    w = rng.standard_normal(3)
    w *= theta / np.linalg.norm(w)
    return np.concatenate([rng.standard_normal(3) * 0.5, w])


def robot(d):
    return oracle.Robot.from_dict(d)


# ---------------------------------------------------------------- FK
def test_fk_orthonormal_30_joints():
    spec, ends = synth.humanoid_robot(103)
    rb = robot(spec)
    assert rb.n_dof == 30
    q = synth.uniform_q(7, 16, rb.dof_lower, rb.dof_upper)
    T = oracle.fk(rb, q)
    R = T.reshape(16, rb.n_joints, 3, 4)[..., :3]
    err = np.abs(np.einsum("...ji,...jk->...ik", R, R) - np.eye(3)).max()
    assert err <= 1e-12
    assert np.abs(np.linalg.det(R) - 1).max() <= 1e-12


def poe_fk(spec, q):
    """Independent FK: product of exponentials of space-frame screw axes taken
    at the home configuration, home frames from plain 4x4 products."""
    n = len(spec["parent"])
    home = []
    for j in range(n):
        O = to44(spec["origin"][j])
        home.append(O if spec["parent"][j] < 0 else home[spec["parent"][j]] @ O)
    screws, v = {}, 0
    var = {}
    for j in range(n):
        if spec["type"][j] == synth.JOINT_FIXED:
            continue
        R, p = home[j][:3, :3], home[j][:3, 3]
        w = R @ spec["axis"][j]
        if spec["type"][j] == synth.JOINT_REVOLUTE:
            screws[j] = np.concatenate([-np.cross(w, p), w])
        else:
            screws[j] = np.concatenate([w, np.zeros(3)])
        var[j] = v
        v += 1
    out = []
    for j in range(n):
        chain = []
        k = j
        while k >= 0:
            chain.append(k)
            k = spec["parent"][k]
        M = np.eye(4)
        for k in reversed(chain):
            if k in screws:
                M = M @ expm(twist_mat(screws[k] * q[var[k]]))
        out.append(to12(M @ home[j]))
    return np.array(out)


@pytest.mark.parametrize("which", ["chain", "prismatic_chain", "hand", "humanoid"])
def test_fk_matches_product_of_exponentials(which):
    if which == "chain":
        spec = synth.chain_robot(100, 7)
    elif which == "prismatic_chain":
        spec = synth.chain_robot(5, 6, prismatic=(1, 4))
    elif which == "hand":
        spec, _ = synth.hand_robot(102)
    else:
        spec, _ = synth.humanoid_robot(103)
    rb = robot(spec)
    qs = synth.uniform_q(11, 5, rb.dof_lower, rb.dof_upper)
    for q in qs:
        np.testing.assert_allclose(oracle.fk(rb, q), poe_fk(spec, q), atol=1e-12, rtol=0)


def one_joint(axis=(0, 0, 1), tool=(1.0, 0, 0), lim=2.8, prismatic=False):
    tool_o = synth.EYE12.copy()
    tool_o[3], tool_o[7], tool_o[11] = tool
    return dict(parent=[-1, 0], type=[2 if prismatic else 1, 0], axis=[axis, (0, 0, 1)],
                origin=[synth.EYE12, tool_o], lower=[-lim, 0], upper=[lim, 0])


def test_single_revolute_textbook():
    rb = robot(one_joint())
    for th in (-2.0, 0.3, 1.7):
        T = oracle.fk(rb, [th])[0].reshape(3, 4)
        c, s = np.cos(th), np.sin(th)
        np.testing.assert_allclose(T[:3, :3], [[c, -s, 0], [s, c, 0], [0, 0, 1]], atol=1e-15)
        T1 = oracle.fk(rb, [th])[1].reshape(3, 4)
        np.testing.assert_allclose(T1[:, 3], [c, s, 0], atol=1e-15)


def test_single_prismatic_textbook():
    rb = robot(one_joint(axis=(0, 1, 0), tool=(0, 0, 0.5), prismatic=True))
    T = oracle.fk(rb, [0.25])[1].reshape(3, 4)
    np.testing.assert_allclose(T[:, 3], [0, 0.25, 0.5], atol=1e-15)
    np.testing.assert_allclose(T[:3, :3], np.eye(3), atol=1e-15)


def planar(l1=0.7, l2=0.4, lim=np.pi):
    o1 = synth.EYE12.copy()
    o2 = synth.EYE12.copy()
    o2[3] = l1
    ot = synth.EYE12.copy()
    ot[3] = l2
    return dict(parent=[-1, 0, 1], type=[1, 1, 0], axis=[(0, 0, 1)] * 3, origin=[o1, o2, ot],
                lower=[-lim, -lim, 0], upper=[lim, lim, 0])


def test_two_link_planar_fk_closed_form():
    l1, l2 = 0.7, 0.4
    rb = robot(planar(l1, l2))
    for q1, q2 in [(0.3, -1.1), (2.0, 0.5), (-1.0, 2.5)]:
        T = oracle.fk(rb, [q1, q2])[2].reshape(3, 4)
        x = l1 * np.cos(q1) + l2 * np.cos(q1 + q2)
        y = l1 * np.sin(q1) + l2 * np.sin(q1 + q2)
        np.testing.assert_allclose(T[:, 3], [x, y, 0], atol=1e-15)
        a = q1 + q2
        np.testing.assert_allclose(T[:2, :2], [[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]],
                                   atol=1e-15)


def test_two_link_planar_lm_reaches_a_closed_form_branch():
    """LM on a position target converges to elbow-up or elbow-down."""
    l1, l2 = 0.7, 0.4
    rb = robot(planar(l1, l2, lim=10.0))
    tg = oracle.Targets([2], [oracle.TARGET_POSITION])
    prm = oracle.IkParams(w_rest=0.0, max_iters=100, tol_pos=1e-12, tol_rot=1.0)
    rng = np.random.default_rng(3)
    for _ in range(6):
        r = rng.uniform(abs(l1 - l2) + 0.05, l1 + l2 - 0.05)
        phi = rng.uniform(-np.pi, np.pi)
        x, y = r * np.cos(phi), r * np.sin(phi)
        T = synth.EYE12.copy()
        T[3], T[7] = x, y
        c2 = (x * x + y * y - l1 * l1 - l2 * l2) / (2 * l1 * l2)
        branches = []
        for s in (+1, -1):
            q2 = s * np.arccos(c2)
            q1 = np.arctan2(y, x) - np.arctan2(l2 * np.sin(q2), l1 + l2 * np.cos(q2))
            branches.append(np.array([q1, q2]))
        seed = rng.uniform(-2, 2, (4, 2))
        out = oracle.ik_solve(rb, prm, tg, T[None, None], seed[None])
        assert out["status"][0] == oracle.P_CONVERGED
        q = out["q"][0]
        wrap = lambda a: (a + np.pi) % (2 * np.pi) - np.pi
        d = min(np.abs(wrap(q - b)).max() for b in branches)
        assert d < 1e-8, (q, branches)


# ---------------------------------------------------------------- SE(3)
def test_se3_exp_log_roundtrip_against_expm():
    rng = np.random.default_rng(0)
    for theta in (0.0, 1e-9, 1e-5, 0.05, 0.0999, 0.1001, 1.0, 2.5, 3.1, np.pi - 1e-4):
        xi = random_twist(rng, theta) if theta > 0 else np.concatenate([rng.standard_normal(3), [0, 0, 0]])
        T = to12(expm(twist_mat(xi)))
        np.testing.assert_allclose(oracle.se3_exp(xi), T, atol=1e-12)
        xi2 = oracle.se3_log(T)
        tol = 1e-7 if theta > np.pi - 1e-3 else 1e-10
        np.testing.assert_allclose(xi2, xi, atol=tol)


def test_se3_log_zero_rotation_is_translation():
    T = synth.EYE12.copy()
    T[3], T[7], T[11] = 0.3, -0.2, 0.9
    np.testing.assert_allclose(oracle.se3_log(T), [0.3, -0.2, 0.9, 0, 0, 0], atol=1e-15)


def test_se3_log_at_pi_reconstructs():
    rng = np.random.default_rng(1)
    for _ in range(5):
        xi = random_twist(rng, np.pi)
        T = to12(expm(twist_mat(xi)))
        xi2 = oracle.se3_log(T)
        assert abs(np.linalg.norm(xi2[3:]) - np.pi) < 1e-7
        np.testing.assert_allclose(to12(expm(twist_mat(xi2))), T, atol=1e-9)


def test_se3_left_jacobian_matches_power_series():
    rng = np.random.default_rng(2)
    for theta in (1e-6, 0.05, 0.2, 1.3, 2.9):
        xi = random_twist(rng, theta)
        A = ad(xi)
        S, term = np.zeros((6, 6)), np.eye(6)
        for k in range(60):
            S += term / _fact(k + 1)
            term = term @ A
        np.testing.assert_allclose(oracle.se3_jl(xi), S, atol=1e-12)
        np.testing.assert_allclose(oracle.se3_jl(xi) @ oracle.se3_jlinv(xi), np.eye(6), atol=1e-11)


def _fact(n):
    out = 1
    for i in range(2, n + 1):
        out *= i
    return out


@pytest.mark.parametrize("theta", [1e-4, 0.05, 0.0999, 0.1001, 0.7, 2.0, 3.0])
def test_se3_jlinv_is_derivative_of_log(theta):
    """d/dh log(exp(h eta) E) at h = 0 equals Jl^-1(log E) eta (central FD)."""
    rng = np.random.default_rng(int(theta * 1e4) + 5)
    xi = random_twist(rng, theta)
    E = expm(twist_mat(xi))
    Jinv = oracle.se3_jlinv(oracle.se3_log(to12(E)))
    h = 1e-6
    for _ in range(3):
        eta = rng.standard_normal(6)
        lp = oracle.se3_log(to12(expm(twist_mat(h * eta)) @ E))
        lm = oracle.se3_log(to12(expm(twist_mat(-h * eta)) @ E))
        fd = (lp - lm) / (2 * h)
        np.testing.assert_allclose(Jinv @ eta, fd, rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------- residuals / Jacobian
def _fd_jacobian(rb, prm, tg, targets, q, h=1e-6):
    m = oracle.n_residuals(rb, tg)
    J = np.zeros((m, rb.n_dof))
    for a in range(rb.n_dof):
        e = np.zeros(rb.n_dof)
        e[a] = h
        rp = oracle.ik_residual(rb, prm, tg, targets, q + e, jacobian=False)
        rm = oracle.ik_residual(rb, prm, tg, targets, q - e, jacobian=False)
        J[:, a] = (rp - rm) / (2 * h)
    return J


def _cases():
    chain = synth.chain_robot(100, 7)
    pchain = synth.chain_robot(9, 6, prismatic=(0, 3))
    hand, tips = synth.hand_robot(102)
    hum, ends = synth.humanoid_robot(103)
    n_chain = len(chain["parent"]) - 1
    return [
        ("chain7", chain, [n_chain], None),
        ("prismatic6", pchain, [len(pchain["parent"]) - 1], None),
        ("hand_positions", hand, list(tips), [oracle.TARGET_POSITION] * 5),
        ("humanoid_poses", hum, list(ends), None),
        ("humanoid_mixed", hum, list(ends), [0, 1, 0, 1, 0, 0]),
    ]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_analytic_jacobian_matches_central_fd(case):
    name, spec, links, kinds = case
    rb = robot(spec)
    tg = oracle.Targets(links, kinds)
    prm = oracle.IkParams()
    rng = np.random.default_rng(4)
    qt = synth.uniform_q(8, 1, rb.dof_lower, rb.dof_upper)[0]
    T = oracle.fk(rb, qt)
    targets = T[links]
    for trial in range(4):
        q = synth.uniform_q(20 + trial, 1, rb.dof_lower, rb.dof_upper)[0]
        if trial == 3:  # push some joints past their limits (away from the kinks)
            q = q.copy()
            q[::3] = rb.dof_upper[::3] + rng.uniform(0.05, 0.3, q[::3].shape)
        r, J = oracle.ik_residual(rb, prm, tg, targets, q)
        Jfd = _fd_jacobian(rb, prm, tg, targets, q)
        scale = np.maximum(1.0, np.abs(J))
        assert np.max(np.abs(J - Jfd) / scale) <= 1e-6, name


def test_pose_jacobian_is_geometric_jacobian_at_solution():
    """At E = I the log derivative is the textbook geometric Jacobian expressed
    in the target frame: [R*^T (w_j x (t* - p_j)); R*^T w_j]."""
    spec = synth.chain_robot(100, 7)
    rb = robot(spec)
    ee = rb.n_joints - 1
    tg = oracle.Targets([ee])
    prm = oracle.IkParams(w_pos=1.0, w_rot=1.0)
    q = synth.uniform_q(31, 1, rb.dof_lower, rb.dof_upper)[0]
    T = oracle.fk(rb, q)
    r, J = oracle.ik_residual(rb, prm, tg, T[[ee]], q)
    Rs = T[ee].reshape(3, 4)[:, :3]
    ts = T[ee].reshape(3, 4)[:, 3]
    G = np.zeros((6, 7))
    for j in range(7):
        Rj = T[j].reshape(3, 4)[:, :3]
        pj = T[j].reshape(3, 4)[:, 3]
        w = Rj @ spec["axis"][j]
        G[:3, j] = Rs.T @ np.cross(w, ts - pj)
        G[3:, j] = Rs.T @ w
    np.testing.assert_allclose(r[:6], 0, atol=1e-12)
    np.testing.assert_allclose(J[:6], G, atol=1e-12)


def test_limit_and_rest_residuals_hand_computed():
    rb = robot(one_joint(lim=2.8))
    tg = oracle.Targets([1])
    prm = oracle.IkParams(w_limit=10.0, w_rest=1e-3)
    T = oracle.fk(rb, [0.0])[[1]]
    for q, hinge in [(3.0, 0.2), (-3.1, 0.3), (1.0, 0.0), (2.8, 0.0)]:
        r, J = oracle.ik_residual(rb, prm, tg, T, [q])
        np.testing.assert_allclose(r[6], 10.0 * hinge, atol=1e-14)
        np.testing.assert_allclose(r[7], 1e-3 * q, atol=1e-15)
        np.testing.assert_allclose(J[6, 0], 10.0 * np.sign(q) * (hinge > 0), atol=0)
        np.testing.assert_allclose(J[7, 0], 1e-3, atol=0)


# ---------------------------------------------------------------- Cholesky / LM
def test_cholesky_matches_lapack():
    rng = np.random.default_rng(5)
    for n in (1, 7, 24, 30):
        M = rng.standard_normal((n, n))
        A = M @ M.T + n * np.eye(n)
        b = rng.standard_normal(n)
        x = oracle.cholesky_solve(A, b)
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)
    assert oracle.cholesky_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.ones(2)) is None


def _config0(batch=16, seeds=1):
    spec = synth.chain_robot(100, 7)
    rb = robot(spec)
    ee = rb.n_joints - 1
    tg = oracle.Targets([ee])
    qt = synth.uniform_q(200, batch, rb.dof_lower, rb.dof_upper)
    targets = oracle.fk(rb, qt)[:, [ee]]
    sd = synth.uniform_q(300, (batch, seeds), rb.dof_lower, rb.dof_upper)
    return rb, tg, targets, sd


def test_first_lm_step_matches_lapack_normal_equations():
    rb, tg, targets, sd = _config0(8)
    prm = oracle.IkParams(max_iters=1)
    out = oracle.ik_solve(rb, prm, tg, targets, sd, n_trace=1)
    for b in range(8):
        q0 = sd[b, 0]
        r, J = oracle.ik_residual(rb, prm, tg, targets[b], q0)
        dq = np.linalg.solve(J.T @ J + 1e-2 * np.eye(7), -J.T @ r)
        rt = oracle.ik_residual(rb, prm, tg, targets[b], q0 + dq, jacobian=False)
        expect = q0 + dq if rt @ rt < r @ r else q0
        np.testing.assert_allclose(out["trace"][b, 0], expect, atol=1e-12)


def test_lm_accepted_costs_strictly_decrease():
    rb, tg, targets, sd = _config0(16)
    prm = oracle.IkParams(max_iters=30)
    out = oracle.ik_solve(rb, prm, tg, targets, sd, n_trace=30)
    for b in range(16):
        prev_q = sd[b, 0]
        prev_f = 0.5 * np.sum(oracle.ik_residual(rb, prm, tg, targets[b], prev_q, jacobian=False) ** 2)
        for t in range(30):
            q = out["trace"][b, t]
            f = 0.5 * np.sum(oracle.ik_residual(rb, prm, tg, targets[b], q, jacobian=False) ** 2)
            if np.array_equal(q, prev_q):
                assert f == prev_f
            else:
                assert f < prev_f
            prev_q, prev_f = q, f


def test_brute_force_one_dof():
    """Global minimum of a 1-DoF position problem found by a dense grid equals
    the best of several LM seeds."""
    L = 0.8
    rb = robot(one_joint(tool=(L, 0, 0), lim=2.8))
    tg = oracle.Targets([1], [oracle.TARGET_POSITION])
    prm = oracle.IkParams(w_rest=0.05, max_iters=200, tol_pos=0.0, tol_rot=0.0)
    target = synth.EYE12.copy()
    target[3], target[7], target[11] = -0.3, 0.5, 0.2
    grid = np.linspace(-3.4, 3.4, 2_000_001)
    hinge = np.maximum(0, grid - 2.8) + np.maximum(0, -2.8 - grid)
    cost = 0.5 * ((L * np.cos(grid) + 0.3) ** 2 + (L * np.sin(grid) - 0.5) ** 2 + 0.2 ** 2) \
        + 0.5 * (10.0 * hinge) ** 2 + 0.5 * (0.05 * grid) ** 2
    q_star = grid[np.argmin(cost)]
    seeds = np.linspace(-2.7, 2.7, 9)[:, None]
    out = oracle.ik_solve(rb, prm, tg, target[None, None], seeds[None])
    assert abs(out["q"][0, 0] - q_star) < 1e-5


def test_best_of_k_selection_rule():
    rb, tg, targets, sd = _config0(32, 8)
    prm = oracle.IkParams(max_iters=15)
    out = oracle.ik_solve(rb, prm, tg, targets, sd, per_problem=True)
    pp = out["per_problem"].reshape(32, 8, -1)
    for b in range(32):
        keys = [(pp[b, s, 11] != 0, pp[b, s, 7], s) for s in range(8)]
        best = min(keys)[2]
        np.testing.assert_array_equal(out["q"][b], pp[b, best, :7])
        assert out["status"][b] == pp[b, best, 11]


def test_multistart_converges_on_reachable_targets():
    rb, tg, targets, sd = _config0(64, 8)
    prm = oracle.IkParams(max_iters=50, early_exit=1)
    out = oracle.ik_solve(rb, prm, tg, targets, sd)
    ok = out["status"] == oracle.P_CONVERGED
    assert ok.mean() >= 0.85  # random-axis chains leave ~2/3 of single seeds in local minima
    assert np.all(out["err"][ok, 0] <= 1e-3) and np.all(out["err"][ok, 1] <= np.deg2rad(0.5))


def test_nonfinite_target_is_flagged():
    rb, tg, targets, sd = _config0(2)
    targets = targets.copy()
    targets[1, 0, 3] = np.nan
    out = oracle.ik_solve(rb, oracle.IkParams(), tg, targets, sd)
    assert out["status"][0] != oracle.P_NONFINITE
    assert out["status"][1] == oracle.P_NONFINITE
