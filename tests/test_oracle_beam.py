"""Pins for the FP64 IK-Beam oracle (Sec. V-C).

IK-Beam is built from the multi-start LM oracle (pinned in test_oracle_pins.py
against closed forms, finite differences, LAPACK and brute force), so each
check below reduces a beam configuration to a case whose answer is fixed
independently of the beam code: one seed split into two phases must follow the
unsplit LM path (the damping carries over), the kept set must be the stable
argsort of the per-seed costs after the first phase, keeping every seed with no
second phase must reproduce the best-of-K rule, and the iteration count must be
the sum of the two phases.
"""
import numpy as np
import pytest

import oracle
from paper_2505_03728_gb300 import synth


@pytest.fixture(scope="module")
def chain():
    spec, qt, _ = synth.ik_workload(synth.IK_PARITY, 12)
    rb = oracle.Robot.from_dict(spec)
    ee = rb.n_joints - 1
    T = oracle.fk(rb, qt)[:, [ee]]
    seeds = synth.uniform_q(41, (12, 16), spec.dof_lower, spec.dof_upper)
    return rb, oracle.Targets([ee]), T, seeds


def test_two_phases_of_one_seed_follow_the_unsplit_lm_path(chain):
    rb, tg, T, seeds = chain
    p = oracle.IkParams(max_iters=0, early_exit=0)
    one = seeds[:, :1]
    for a, b in ((0, 9), (3, 6), (6, 10)):
        beam = oracle.ik_beam(rb, p, tg, T, one, steps1=a, keep=1, steps2=b)
        ref = oracle.ik_solve(rb, oracle.IkParams(max_iters=a + b, early_exit=0), tg, T, one)
        np.testing.assert_allclose(beam["q"], ref["q"], rtol=0, atol=1e-12)
        np.testing.assert_array_equal(beam["iters"], ref["iters"])
        np.testing.assert_array_equal(beam["status"], ref["status"])


def test_damping_carries_over_between_phases(chain):
    """Restarting the damping at lambda0 in the second phase changes the path
    (the check above would then fail); this confirms the case is sensitive."""
    rb, tg, T, seeds = chain
    one = seeds[:, :1]
    p6 = oracle.IkParams(max_iters=6, early_exit=0)
    first = oracle.ik_solve(rb, p6, tg, T, one)
    restarted = oracle.ik_solve(rb, oracle.IkParams(max_iters=6, early_exit=0), tg, T, first["q"][:, None])
    ref = oracle.ik_solve(rb, oracle.IkParams(max_iters=12, early_exit=0), tg, T, one)
    beam = oracle.ik_beam(rb, p6, tg, T, one, steps1=6, keep=1, steps2=6)
    assert np.abs(restarted["q"] - ref["q"]).max() > 1e-9
    np.testing.assert_allclose(beam["q"], ref["q"], rtol=0, atol=1e-12)


def test_kept_seeds_are_the_stable_argsort_of_phase_one_costs(chain):
    rb, tg, T, seeds = chain
    B, S = seeds.shape[:2]
    p = oracle.IkParams(max_iters=6, early_exit=0)
    per = oracle.ik_solve(rb, p, tg, T, seeds, per_problem=True)["per_problem"]
    cost = per[:, rb.n_dof].reshape(B, S)
    cost = np.where(np.isfinite(cost), cost, np.inf)
    beam = oracle.ik_beam(rb, p, tg, T, seeds, steps1=6, keep=4, steps2=0)
    for b in range(B):
        np.testing.assert_array_equal(beam["kept"][b], np.argsort(cost[b], kind="stable")[:4])


def test_keeping_every_seed_without_a_second_phase_is_multistart(chain):
    rb, tg, T, seeds = chain
    S = seeds.shape[1]
    p = oracle.IkParams(max_iters=7, early_exit=0)
    beam = oracle.ik_beam(rb, p, tg, T, seeds, steps1=7, keep=S, steps2=0)
    ref = oracle.ik_solve(rb, p, tg, T, seeds)
    np.testing.assert_allclose(beam["q"], ref["q"], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(beam["status"], ref["status"])
    np.testing.assert_allclose(beam["err"], ref["err"], rtol=0, atol=1e-12)


def test_iterations_add_up_and_early_exit_stops_both_phases(chain):
    rb, tg, T, seeds = chain
    fixed = oracle.ik_beam(rb, oracle.IkParams(early_exit=0), tg, T, seeds, steps1=6, keep=4, steps2=10)
    assert np.all(fixed["iters"] == 16)
    early = oracle.ik_beam(rb, oracle.IkParams(early_exit=1), tg, T, seeds, steps1=6, keep=4, steps2=10)
    assert np.all(early["iters"] <= 16)
    conv = early["status"] == 0
    assert np.all(early["err"][conv, 0] <= 1e-3) and np.all(early["err"][conv, 1] <= np.deg2rad(0.5))
    assert conv.mean() >= 0.75  # 16 seeds, 4 kept: most reachable targets are solved
