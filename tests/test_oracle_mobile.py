"""Mobile-base IK (Sec. V-B): the SE(2) base as prismatic x, prismatic y and
revolute z joints ahead of the arm.  Pinned against the closed form
T_world<-base(x, y, theta) T_base<-i of the arm's own FK."""
import numpy as np

import oracle
from paper_2505_03728_gb300 import synth


def planar(x, y, th):
    c, s = np.cos(th), np.sin(th)
    M = np.eye(4)
    M[:2, :2] = [[c, -s], [s, c]]
    M[0, 3], M[1, 3] = x, y
    return M


def to44(T12):
    M = np.eye(4)
    M[:3, :] = np.asarray(T12).reshape(3, 4)
    return M


def test_mobile_fk_is_base_transform_times_arm_fk():
    arm, mob, qt, shift, _ = synth.mobile_workload(batch=16)
    oa, om = oracle.Robot.from_dict(arm), oracle.Robot.from_dict(mob)
    rng = np.random.default_rng(3)
    base = np.column_stack([rng.uniform(-3, 3, 16), rng.uniform(-3, 3, 16), rng.uniform(-4, 4, 16)])
    Ta = oracle.fk(oa, qt)
    Tm = oracle.fk(om, np.hstack([base, qt]))
    for b in range(16):
        P = planar(*base[b])
        for j in range(oa.n_joints):
            np.testing.assert_allclose(to44(Tm[b, j + 3]), P @ to44(Ta[b, j]), atol=1e-12)


def test_mobile_ik_reaches_shifted_targets_the_fixed_base_cannot():
    """The oracle's LM on a few shifted targets: with the base as variables the
    targets are reached at 5 mm / 0.05 rad; the fixed arm mostly cannot."""
    cfg = dict(synth.MOBILE, batch=24, n_seeds=4)
    arm, mob, qt, shift, sd = synth.mobile_workload(cfg)
    oa, om = oracle.Robot.from_dict(arm), oracle.Robot.from_dict(mob)
    ee = oa.n_joints - 1
    T = oracle.fk(oa, qt)[:, ee].copy()
    T[:, 3] += shift[:, 0]
    T[:, 7] += shift[:, 1]
    prm = oracle.IkParams(max_iters=50, early_exit=1, tol_pos=5e-3, tol_rot=0.05)
    fixed = oracle.ik_solve(oa, prm, oracle.Targets([ee]), T[:, None], sd)
    seeds_m = np.concatenate([np.zeros(sd.shape[:2] + (3,)), sd], axis=2)
    mobile = oracle.ik_solve(om, prm, oracle.Targets([ee + 3]), T[:, None], seeds_m)
    assert (mobile["status"] == 0).mean() >= 0.9
    assert (mobile["status"] == 0).mean() >= (fixed["status"] == 0).mean() + 0.3
