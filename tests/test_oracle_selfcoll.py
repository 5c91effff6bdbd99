"""Self-collision cost of the oracle (Sec. III-C with Eq. 1): one residual row
per sphere pair, w_self f(|c_a - c_b| - r_a - r_b, eta), sphere centres riding
on joint frames.  Pinned by recomputing the distances from the oracle's own FK
frames in numpy (a plain re-derivation of the geometry), against Eq. 1's
closed form, and by central differences of the full residual vector (rows away
from the activation's kinks), with and without mimic joints."""
import numpy as np

import oracle
from paper_2505_03728_gb300 import synth


def f_eta(d, eta):
    return np.where(d <= 0, -d + 0.5 * eta, np.where(d < eta, 0.5 / eta * (eta - d) ** 2, 0.0))


def robot(mimic):
    spec, tips = synth.hand_mimic_robot() if mimic else synth.hand_robot(102)
    spec = dict(spec)
    spec["spheres"] = synth.hand_collision_spheres(spec, tips, radius=0.02)
    return spec, oracle.Robot.from_dict(spec), list(tips)


def centres(o, sp, q):
    T = oracle.fk(o, q[None])[0].reshape(-1, 3, 4)
    return np.stack([T[j, :, :3] @ c + T[j, :, 3] for j, c in zip(sp["joint"], sp["centre"])])


def test_rows_are_eq1_of_the_sphere_distances():
    spec, o, tips = robot(False)
    sp = spec["spheres"]
    prm = oracle.IkParams(w_self=7.0, eta_self=0.03)
    tg = oracle.Targets(tips, [1] * 5)
    T = oracle.fk(o, synth.uniform_q(1, 1, o.dof_lower, o.dof_upper))[0][tips]
    n_active = 0
    for trial in range(20):
        q = synth.uniform_q(100 + trial, 1, o.dof_lower, o.dof_upper)[0]
        r, _ = oracle.ik_residual(o, prm, tg, T, q)
        c = centres(o, sp, q)
        a, b = sp["pairs"][:, 0], sp["pairs"][:, 1]
        d = np.linalg.norm(c[a] - c[b], axis=1) - sp["radius"][a] - sp["radius"][b]
        np.testing.assert_allclose(r[-len(a):], 7.0 * f_eta(d, 0.03), atol=1e-12)
        n_active += int(np.sum(d < 0.03))
    assert n_active > 0  # some pairs come within the buffer


def test_jacobian_matches_central_differences():
    for mimic in (False, True):
        spec, o, tips = robot(mimic)
        sp = spec["spheres"]
        prm = oracle.IkParams(w_self=5.0, eta_self=0.03)
        tg = oracle.Targets(tips, [1, 0, 1, 0, 1])
        T = oracle.fk(o, synth.uniform_q(2, 1, o.dof_lower, o.dof_upper))[0][tips]
        checked = 0
        for trial in range(25):
            q = synth.uniform_q(200 + trial, 1, o.dof_lower, o.dof_upper)[0]
            r, J = oracle.ik_residual(o, prm, tg, T, q)
            c = centres(o, sp, q)
            a, b = sp["pairs"][:, 0], sp["pairs"][:, 1]
            d = np.linalg.norm(c[a] - c[b], axis=1) - sp["radius"][a] - sp["radius"][b]
            smooth = (np.abs(d) > 1e-4) & (np.abs(d - 0.03) > 1e-4)
            h = 1e-6
            fd = np.zeros_like(J)
            for v in range(o.n_dof):
                dq = np.zeros(o.n_dof)
                dq[v] = h
                fd[:, v] = (oracle.ik_residual(o, prm, tg, T, q + dq)[0] - oracle.ik_residual(o, prm, tg, T, q - dq)[0]) / (2 * h)
            rows = np.arange(len(r) - len(a), len(r))[smooth]
            err = np.abs(fd[rows] - J[rows]) / np.maximum(1.0, np.abs(J[rows]))
            assert err.max() <= 1e-6, (mimic, trial, err.max())
            checked += int(np.sum(smooth & (d < 0.03)))
        assert checked > 0


def test_no_pairs_no_rows():
    spec, tips = synth.hand_robot(102)
    o = oracle.Robot.from_dict(spec)
    tg = oracle.Targets(list(tips), [1] * 5)
    assert oracle.n_residuals(o, tg) == 15 + 2 * 24
