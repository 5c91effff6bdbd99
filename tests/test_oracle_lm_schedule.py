"""Pins for the oracle's Levenberg-Marquardt damping schedule (Sec. III-A) and
its success measure, against an independent re-derivation.

Sec. III-A names Levenberg-Marquardt and nothing more; the readings fixed for
this build are: damping D = I, lambda0 = 1e-2, accept a trial iff the cost
strictly decreases, lambda / nu on accept and lambda * nu on reject, clamped
to [lambda_min, lambda_max], a rejected iteration counts toward the iteration
cap, and the convergence test (position <= tol_pos and rotation angle <=
tol_rot for every target) runs before the first iteration and after every
accepted step.

Each test below runs the same rules in a plain numpy loop that shares nothing
with the oracle's C loop: residuals and Jacobians come from
``oracle.ik_residual`` (pinned by central differences and closed forms in
test_oracle_pins.py), the damped step from LAPACK (``numpy.linalg.solve``),
the pose errors from a ``scipy.spatial.transform.Rotation`` angle and a plain
vector norm.  The oracle's iterates and its damping after every iteration
must agree with the loop: flipping nu, dropping either clamp or not counting
a rejected iteration each fails one of the named tests.  The success measure
(``oracle.ik_errors``) is pinned separately by poses built with a known
translation offset and a known rotation angle.
"""
import numpy as np
import pytest
from scipy.linalg import expm
from scipy.spatial.transform import Rotation

import oracle
from paper_2505_03728_gb300 import synth

TIE = 1e-9  # relative cost change below which FP64 rounding may flip an accept


def _hat(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]], dtype=float)


def _chain(batch, seeds=1, target_seed=200, seed_seed=300):
    spec = synth.chain_robot(100, 7)
    rb = oracle.Robot.from_dict(spec)
    ee = rb.n_joints - 1
    tg = oracle.Targets([ee])
    qt = synth.uniform_q(target_seed, batch, rb.dof_lower, rb.dof_upper)
    targets = oracle.fk(rb, qt)[:, [ee]]
    sd = synth.uniform_q(seed_seed, (batch, seeds), rb.dof_lower, rb.dof_upper)
    return rb, tg, targets, sd


def _errors(rb, tg, targets, q):
    """max over targets of |t - t*| and of the angle of R*^T R (scipy)."""
    T = oracle.fk(rb, q)
    pe = re = 0.0
    for k in range(tg.k):
        Tl = T[tg.links[k]].reshape(3, 4)
        Tt = np.asarray(targets[k]).reshape(3, 4)
        pe = max(pe, float(np.linalg.norm(Tl[:, 3] - Tt[:, 3])))
        if tg.kinds is None or tg.kinds[k] == oracle.TARGET_POSE:
            re = max(re, float(Rotation.from_matrix(Tt[:, :3].T @ Tl[:, :3]).magnitude()))
    return pe, re


def numpy_lm(rb, prm, tg, targets, seed, lam_init=None):
    """The LM rules written out with LAPACK; returns (q after each iteration,
    damping after each iteration, accepted flags, iterations, converged,
    index of the first near-tie iteration or None)."""
    n = rb.n_dof
    q = np.array(seed, dtype=float)
    lam = prm.lambda0 if lam_init is None else lam_init
    r = oracle.ik_residual(rb, prm, tg, targets, q, jacobian=False)
    f = 0.5 * r @ r

    def conv_of(qq):
        pe, re = _errors(rb, tg, targets, qq)
        return pe <= prm.tol_pos and re <= prm.tol_rot

    conv = conv_of(q)
    qs, lams, acc, tie = [], [], [], None
    it = 0
    if not (prm.early_exit and conv):
        while it < prm.max_iters:
            it += 1
            r, J = oracle.ik_residual(rb, prm, tg, targets, q)
            A = J.T @ J + lam * np.eye(n)
            accepted = False
            try:
                np.linalg.cholesky(A)
                spd = True
            except np.linalg.LinAlgError:
                spd = False
            if spd:
                qt = q + np.linalg.solve(A, -(J.T @ r))
                rt = oracle.ik_residual(rb, prm, tg, targets, qt, jacobian=False)
                ft = 0.5 * rt @ rt
                if tie is None and abs(ft - f) <= TIE * f:
                    tie = it
                if ft < f:
                    accepted, q, f = True, qt, ft
            if accepted:
                lam = max(lam / prm.nu, prm.lambda_min)
                conv = conv_of(q)
            else:
                lam = min(lam * prm.nu, prm.lambda_max)
            qs.append(q.copy())
            lams.append(lam)
            acc.append(accepted)
            if prm.early_exit and conv:
                break
    return np.array(qs).reshape(-1, n), np.array(lams), np.array(acc, bool), it, conv, tie


def _compare(rb, prm, tg, targets, seeds, lam_init=None, atol=1e-11):
    """Run the oracle and the numpy loop on every problem; assert agreement up
    to the first near-tie and return the accept flags.  Near-ties (a cost
    change below 1e-9 relative, where rounding decides the accept) only come
    once a run sits at a stationary point, never in the first five
    iterations, and leave most iterations compared."""
    all_acc, ties, compared, total = [], 0, 0, 0
    for b in range(len(seeds)):
        kw = {} if lam_init is None else dict(lambda_init=lam_init)
        o = oracle.lm_run(rb, prm, tg, targets[b], seeds[b], prm.max_iters, **kw)
        qs, lams, acc, it, conv, tie = numpy_lm(rb, prm, tg, targets[b], seeds[b], lam_init)
        upto = it if tie is None else tie - 1
        ties += tie is not None
        assert tie is None or tie > 5
        compared += upto
        total += it
        np.testing.assert_allclose(o["q_trace"][:upto], qs[:upto], rtol=0, atol=atol)
        np.testing.assert_array_equal(o["lam_trace"][:upto], lams[:upto])
        if tie is None:
            assert o["iters"] == it
            assert (o["status"] == oracle.P_CONVERGED) == conv
            np.testing.assert_allclose(o["q"], qs[-1] if it else seeds[b], rtol=0, atol=atol)
        all_acc.append(acc[:upto])
    assert compared >= 0.75 * total, (compared, total, ties)
    return all_acc


# ---------------------------------------------------------------- damping schedule
def test_lm_trace_and_damping_match_numpy_rederivation():
    rb, tg, targets, sd = _chain(16)
    prm = oracle.IkParams(max_iters=30, early_exit=0)
    acc = _compare(rb, prm, tg, targets, sd[:, 0])
    flat = np.concatenate(acc)
    # both branches of the damping rule are exercised
    assert flat.sum() >= 50 and (~flat).sum() >= 10


def test_lm_early_exit_iteration_counts_match():
    rb, tg, targets, sd = _chain(16, target_seed=210, seed_seed=310)
    prm = oracle.IkParams(max_iters=50, early_exit=1)
    _compare(rb, prm, tg, targets, sd[:, 0])


@pytest.mark.parametrize("nu", [3.0, 1.5])
def test_nu_is_the_damping_factor(nu):
    rb, tg, targets, sd = _chain(6, target_seed=220, seed_seed=320)
    prm = oracle.IkParams(max_iters=20, nu=nu)
    _compare(rb, prm, tg, targets, sd[:, 0])
    o = oracle.lm_run(rb, prm, tg, targets[0], sd[0, 0], 20)
    lam = np.concatenate([[prm.lambda0], o["lam_trace"]])
    ratio = lam[1:] / lam[:-1]
    # every update multiplies or divides by nu (no clamp is reached here)
    assert np.all(np.isclose(ratio, nu, rtol=1e-15) | np.isclose(ratio, 1 / nu, rtol=1e-15))


def test_lambda_min_clamp():
    """lambda0 = lambda_min: every accept would lower the damping, the clamp
    keeps it at the floor."""
    rb, tg, targets, sd = _chain(8, target_seed=230, seed_seed=330)
    prm = oracle.IkParams(max_iters=25, lambda0=1e-2, lambda_min=1e-2)
    acc = _compare(rb, prm, tg, targets, sd[:, 0])
    hits = 0
    for b in range(8):
        o = oracle.lm_run(rb, prm, tg, targets[b], sd[b, 0], 25)
        assert o["lam_trace"].min() == 1e-2
        lam_prev = np.concatenate([[1e-2], o["lam_trace"][:-1]])
        hits += int(np.sum(acc[b] & (lam_prev[:len(acc[b])] == 1e-2)))
    assert hits >= 10  # accepts taken at the floor


def test_lambda_max_clamp():
    """lambda0 = lambda_max: every reject would raise the damping, the clamp
    keeps it at the ceiling."""
    rb, tg, targets, sd = _chain(8, target_seed=240, seed_seed=340)
    prm = oracle.IkParams(max_iters=25, lambda0=1e-6, lambda_max=1e-6, lambda_min=1e-12)
    acc = _compare(rb, prm, tg, targets, sd[:, 0])
    hits = 0
    for b in range(8):
        o = oracle.lm_run(rb, prm, tg, targets[b], sd[b, 0], 25)
        assert o["lam_trace"].max() == 1e-6
        lam_prev = np.concatenate([[1e-6], o["lam_trace"][:-1]])
        hits += int(np.sum(~acc[b] & (lam_prev[:len(acc[b])] == 1e-6)))
    assert hits >= 3  # rejects taken at the ceiling


def test_rejected_iterations_count_toward_the_cap():
    """With a tiny damping most early trials overshoot and are rejected; every
    problem that has not converged stops after exactly max_iters iterations,
    rejected ones included, and its iterate is unchanged by the rejects."""
    rb, tg, targets, sd = _chain(16, target_seed=250, seed_seed=350)
    prm = oracle.IkParams(max_iters=4, early_exit=1, lambda0=1e-9, lambda_min=1e-10)
    # at lambda ~ 1e-9 the damped normal matrix has a condition number near
    # 1e9, so LAPACK's and the oracle's Cholesky steps differ by ~eps * 1e9
    acc = _compare(rb, prm, tg, targets, sd[:, 0], atol=1e-6)
    rejected_then_capped = 0
    for b in range(16):
        o = oracle.lm_run(rb, prm, tg, targets[b], sd[b, 0], 4)
        if o["status"] != oracle.P_CONVERGED:
            assert o["iters"] == 4
            rejected_then_capped += int((~acc[b]).any())
        for k in np.flatnonzero(~acc[b]):
            prev = sd[b, 0] if k == 0 else o["q_trace"][k - 1]
            np.testing.assert_array_equal(o["q_trace"][k], prev)
    assert rejected_then_capped >= 3


def test_damping_carried_into_a_continued_run():
    """An LM run continued from a stored damping (the IK-Beam second round)
    follows the same rules from that damping."""
    rb, tg, targets, sd = _chain(6, target_seed=260, seed_seed=360)
    prm = oracle.IkParams(max_iters=10)
    _compare(rb, prm, tg, targets, sd[:, 0], lam_init=0.37)


# ---------------------------------------------------------------- success measure
def test_ik_errors_recover_known_offsets_and_angles():
    """Targets built from the link frame by a translation of known length and a
    rotation of known angle about a random axis: the oracle's errors are that
    length and that angle, from 0 up to within 1e-9 of pi."""
    rb, tg, _, _ = _chain(1)
    rng = np.random.default_rng(11)
    ee = tg.links[0]
    angles = [0.0, 1e-12, 1e-9, 1e-6, 1e-3, 0.1, 0.5, 1.0, 2.0, 3.0, np.pi - 1e-3, np.pi - 1e-6, np.pi - 1e-9]
    for i, th in enumerate(angles):
        q = rng.uniform(-2.8, 2.8, rb.n_dof)
        Tl = oracle.fk(rb, q)[ee].reshape(3, 4)
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        d = rng.standard_normal(3)
        length = [0.0, 1e-7, 1e-3, 0.3][i % 4]
        d *= length / np.linalg.norm(d)
        Tt = np.zeros((3, 4))
        Tt[:, :3] = Tl[:, :3] @ expm(_hat(a * th))
        Tt[:, 3] = Tl[:, 3] + d
        pe, re = oracle.ik_errors(rb, tg, Tt.reshape(1, 12), q)
        assert abs(pe - length) <= 1e-15 + 1e-12 * length
        assert abs(re - th) <= 2e-12, (th, re)


def test_ik_errors_take_the_maximum_over_targets_and_skip_rotation_of_position_targets():
    spec, ends = synth.hand_robot(102)
    rb = oracle.Robot.from_dict(spec)
    k = len(ends)
    rng = np.random.default_rng(12)
    q = rng.uniform(rb.dof_lower, rb.dof_upper)
    T = oracle.fk(rb, q)
    lengths = rng.uniform(0.0, 0.05, k)
    tgts = []
    for j, e in enumerate(ends):
        M = T[e].reshape(3, 4).copy()
        d = rng.standard_normal(3)
        M[:, 3] += d * lengths[j] / np.linalg.norm(d)
        M[:, :3] = M[:, :3] @ expm(_hat(rng.standard_normal(3)))  # ignored by position targets
        tgts.append(M.reshape(12))
    tg = oracle.Targets(ends, [oracle.TARGET_POSITION] * k)
    pe, re = oracle.ik_errors(rb, tg, np.array(tgts), q)
    assert abs(pe - lengths.max()) <= 1e-14 and re == 0.0
    # as pose targets the rotation error is the largest angle, measured by scipy
    tg = oracle.Targets(ends)
    pe, re = oracle.ik_errors(rb, tg, np.array(tgts), q)
    pe2, re2 = _errors(rb, tg, np.array(tgts), q)
    assert abs(pe - pe2) <= 1e-14 and abs(re - re2) <= 1e-12


def test_ik_errors_against_scipy_on_random_pose_pairs():
    rb, tg, _, _ = _chain(1)
    rng = np.random.default_rng(13)
    ee = tg.links[0]
    for _ in range(200):
        q1, q2 = rng.uniform(-2.8, 2.8, (2, rb.n_dof))
        target = oracle.fk(rb, q2)[ee]
        pe, re = oracle.ik_errors(rb, tg, target[None], q1)
        pe2, re2 = _errors(rb, tg, target[None], q1)
        assert abs(pe - pe2) <= 1e-14 and abs(re - re2) <= 1e-12


# ---------------------------------------------------------------- trajectory LM
def _traj_small(T=8, seed=1):
    spec = synth.chain_robot(100, 7)
    rb = oracle.Robot.from_dict(spec)
    rng = np.random.default_rng(seed)
    qs = synth.uniform_q(seed + 11, 1, rb.dof_lower, rb.dof_upper)[0]
    qg = synth.uniform_q(seed + 12, 1, rb.dof_lower, rb.dof_upper)[0]
    x = synth.linear_interpolation(qs[None], qg[None], T)[0] + rng.normal(0, 0.05, (T, 7))
    Tf = oracle.fk(rb, x[T // 2])
    obs = [[*(Tf[j].reshape(3, 4)[:, 3] + rng.normal(0, 0.05, 3)), 0.1] for j in (2, 4, 6)]
    scene = oracle.Scene(synth.link_spheres(3, 7), np.array(obs), [0, 0, 1, -0.15])
    return rb, scene, x, qs, oracle.fk(rb, qg)[-1]


def numpy_traj_lm(rb, prm, scene, x0, qs, goal):
    """The trajectory LM with the IK rules: normal equations from
    oracle.traj_normal (pinned as J^T J of the finite-difference-checked
    Jacobian), the damped step from LAPACK."""
    x = np.array(x0, dtype=float)
    lam = prm.lambda0
    f, A, g = oracle.traj_normal(rb, prm, scene, x, qs, goal)
    xs, lams, tie = [], [], None
    for it in range(prm.iters):
        Al = A + lam * np.eye(A.shape[0])
        accepted = False
        try:
            np.linalg.cholesky(Al)
            spd = True
        except np.linalg.LinAlgError:
            spd = False
        if spd:
            xt = x + np.linalg.solve(Al, -g).reshape(x.shape)
            ft = oracle.traj_normal(rb, prm, scene, xt, qs, goal)[0]
            if tie is None and abs(ft - f) <= TIE * f:
                tie = it
            if ft < f:
                accepted, x = True, xt
                f, A, g = oracle.traj_normal(rb, prm, scene, x, qs, goal)
        lam = max(lam / prm.nu, prm.lambda_min) if accepted else min(lam * prm.nu, prm.lambda_max)
        xs.append(x.copy())
        lams.append(lam)
    return np.array(xs), np.array(lams), tie


@pytest.mark.parametrize("banded", [1, 0])
@pytest.mark.parametrize("lam", [dict(), dict(lambda0=1e-2, lambda_min=1e-2), dict(lambda0=1e-4, lambda_max=1e-4)])
def test_traj_lm_trace_and_damping_match_numpy_rederivation(banded, lam):
    rb, scene, x, qs, goal = _traj_small()
    prm = oracle.TrajParams(iters=20, banded=banded, **lam)
    o = oracle.traj_lm_run(rb, prm, scene, x, qs, goal)
    xs, lams, tie = numpy_traj_lm(rb, prm, scene, x, qs, goal)
    upto = prm.iters if tie is None else tie
    np.testing.assert_allclose(o["trace"][:upto], xs[:upto], rtol=0, atol=1e-9)
    np.testing.assert_array_equal(o["lam_trace"][:upto], lams[:upto])
    steps = np.concatenate([[prm.lambda0], lams])
    up, down = np.sum(steps[1:] > steps[:-1]), np.sum(steps[1:] < steps[:-1])
    if not lam:
        assert up >= 1 and down >= 5  # both branches exercised
    else:
        clamp = lam.get("lambda_min", lam.get("lambda_max"))
        assert np.any(lams == clamp) and (lams.min() >= clamp if "lambda_min" in lam else lams.max() <= clamp)
