"""Mimic joints (Sec. III-B): a joint that follows another joint's variable,
value = m q_source + o.  Pinned by expanding to the plain robot (every joint
its own variable) with the mimic values substituted, and by the chain rule
for the Jacobian: J_mimic = J_plain E, E mapping the reduced variables to the
full ones (E = 1 for a joint's own variable, m for its mimic followers) --
with J_plain itself pinned against central differences in test_oracle_pins."""
import numpy as np

import oracle
from paper_2505_03728_gb300 import synth


def expand(spec, q_red):
    """Full joint values of the plain robot for reduced variables q_red."""
    t = np.asarray(spec["type"])
    mimic = np.asarray(spec["mimic"])
    own = (t != 0) & (mimic < 0)
    red_index = -np.ones(len(t), int)
    red_index[own] = np.arange(own.sum())
    movable = np.nonzero(t != 0)[0]
    q_full = np.zeros(q_red.shape[:-1] + (len(movable),))
    E = np.zeros((len(movable), own.sum()))
    for f, j in enumerate(movable):
        if mimic[j] >= 0:
            s = mimic[j]
            q_full[..., f] = spec["mimic_mult"][j] * q_red[..., red_index[s]] + spec["mimic_off"][j]
            E[f, red_index[s]] = spec["mimic_mult"][j]
        else:
            q_full[..., f] = q_red[..., red_index[j]]
            E[f, red_index[j]] = 1.0
    return q_full, E


def plain(spec):
    d = {k: spec[k] for k in ("parent", "type", "axis", "origin", "lower", "upper")}
    return oracle.Robot.from_dict(d)


def test_mimic_hand_has_five_fewer_variables():
    spec, tips = synth.hand_mimic_robot()
    assert oracle.Robot.from_dict(spec).n_dof == 19 == spec.n_dof
    assert plain(spec).n_dof == 24


def test_mimic_fk_equals_plain_fk_with_substituted_values():
    spec, tips = synth.hand_mimic_robot()
    om, op = oracle.Robot.from_dict(spec), plain(spec)
    q = synth.uniform_q(3, 20, om.dof_lower, om.dof_upper)
    qf, _ = expand(spec, q)
    np.testing.assert_allclose(oracle.fk(om, q), oracle.fk(op, qf), atol=1e-13)


def test_mimic_jacobian_is_the_chain_rule_of_the_plain_jacobian():
    spec, tips = synth.hand_mimic_robot()
    om, op = oracle.Robot.from_dict(spec), plain(spec)
    links = list(tips)
    for kinds in ([1] * 5, [0, 1, 0, 1, 0]):
        tg = oracle.Targets(links, kinds)
        prm = oracle.IkParams()
        rng = np.random.default_rng(4)
        for trial in range(5):
            q = synth.uniform_q(10 + trial, 1, om.dof_lower, om.dof_upper)[0]
            qf, E = expand(spec, q)
            T = oracle.fk(op, synth.uniform_q(20 + trial, 1, op.dof_lower, op.dof_upper))[0][links]
            rm, Jm = oracle.ik_residual(om, prm, tg, T, q)
            rp, Jp = oracle.ik_residual(op, prm, tg, T, qf)
            npose = sum(6 if k == 0 else 3 for k in kinds)
            np.testing.assert_allclose(rm[:npose], rp[:npose], atol=1e-13)
            np.testing.assert_allclose(Jm[:npose], Jp[:npose] @ E, atol=1e-12)
            # central differences of the mimic robot's own residual
            h = 1e-6
            fd = np.zeros_like(Jm)
            for v in range(om.n_dof):
                dq = np.zeros(om.n_dof)
                dq[v] = h
                fd[:, v] = (oracle.ik_residual(om, prm, tg, T, q + dq)[0] - oracle.ik_residual(om, prm, tg, T, q - dq)[0]) / (2 * h)
            assert np.abs(fd[:npose] - Jm[:npose]).max() <= 1e-6 * max(1.0, np.abs(Jm).max())
