"""Self-collision cost on the GPU (Sec. III-C, Eq. 1): sphere pairs of a hand
(neighbouring fingers' links) as residual rows of the warp-per-problem solver,
against the FP64 oracle (pinned in test_oracle_selfcoll.py)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_03728_gb300 import build, pk, synth

pytestmark = pytest.mark.gpu

W_SELF, ETA = 10.0, 0.03


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def oparams(p):
    return oracle.IkParams(w_pos=p.w_pos, w_rot=p.w_rot, w_limit=p.w_limit, w_rest=p.w_rest, lambda0=p.lambda0,
                           lambda_min=p.lambda_min, lambda_max=p.lambda_max, nu=p.nu, tol_pos=p.tol_pos,
                           tol_rot=p.tol_rot, max_iters=p.max_iters, early_exit=p.early_exit, w_self=p.w_self,
                           eta_self=p.eta_self)


def setup(mimic, B, S, seed=0):
    spec, tips = synth.hand_mimic_robot() if mimic else synth.hand_robot(102)
    spec = synth.RobotSpec(spec)
    spec["spheres"] = synth.hand_collision_spheres(spec, tips, radius=0.02)
    g, o = pk.Robot.from_spec(spec), oracle.Robot.from_dict(spec)
    links = list(tips)
    qt = synth.uniform_q(950 + seed, B, o.dof_lower, o.dof_upper)
    T = oracle.fk(o, qt)[:, links]
    sd = synth.uniform_q(960 + seed, (B, S), o.dof_lower, o.dof_upper)
    return spec, g, o, links, T, sd


def min_distance(o, spec, q):
    sp = spec["spheres"]
    Tf = oracle.fk(o, q).reshape(q.shape[0], -1, 3, 4)
    c = np.stack([np.einsum("bij,j->bi", Tf[:, j, :, :3], cc) + Tf[:, j, :, 3]
                  for j, cc in zip(sp["joint"], sp["centre"])], axis=1)
    a, b = sp["pairs"][:, 0], sp["pairs"][:, 1]
    d = np.linalg.norm(c[:, a] - c[:, b], axis=2) - sp["radius"][a] - sp["radius"][b]
    return d.min(axis=1)


@pytest.mark.parametrize("mimic", [False, True], ids=["hand24", "hand24_mimic"])
def test_self_collision_iterates_match_oracle(mimic):
    spec, g, o, links, T, sd = setup(mimic, 97, 1)
    kinds = [pk.PK_TARGET_POSITION] * 5
    tg = oracle.Targets(links, kinds)
    base = pk.pk_ik_params_default(max_iters=5, early_exit=0, w_self=W_SELF, eta_self=ETA)
    ref = oracle.ik_solve(o, oparams(base), tg, T, sd, n_trace=5)
    tie = ref["margin"] <= 1e-5
    assert (min_distance(o, spec, sd[:, 0]) < ETA).mean() >= 0.2  # the cost is active on many seeds
    for k in range(1, 6):
        p = pk.pk_ik_params_default(max_iters=k, early_exit=0, w_self=W_SELF, eta_self=ETA)
        q = pk.pk_ik_solve(g, p, links, kinds, dev(T), dev(sd))[0].cpu().numpy().astype(np.float64)
        qr = ref["trace"][:, k - 1]
        rel = (np.abs(q - qr) / np.maximum(1.0, np.abs(qr))).max(axis=1)
        assert np.all(rel[~tie] <= 1e-4), (mimic, k, np.sort(rel)[-4:])
    assert tie.sum() <= 5


def test_self_collision_cost_separates_the_fingers():
    spec, g, o, links, T, sd = setup(False, 512, 4, seed=1)
    kinds = [pk.PK_TARGET_POSITION] * 5
    out = {}
    for w in (0.0, W_SELF):
        p = pk.pk_ik_params_default(max_iters=50, early_exit=0, w_self=w, eta_self=ETA)
        q = pk.pk_ik_solve(g, p, links, kinds, dev(T), dev(sd))[0].cpu().numpy().astype(np.float64)
        out[w] = min_distance(o, spec, q)
    pen0, pen1 = (out[0.0] < 0).mean(), (out[W_SELF] < 0).mean()
    print(f"solutions with penetrating finger spheres: without the cost {pen0:.3f}, with it {pen1:.3f}")
    assert pen1 < 0.5 * pen0


def test_self_collision_leaves_the_chain_kernels():
    spec = synth.chain_robot(100, 7)
    g = pk.Robot.from_spec(spec)
    g.set_spheres([2, 6], [[0, 0, 0.05], [0, 0, 0.05]], [0.05, 0.05], [[0, 1]])
    ee = g.n_joints - 1
    T = pk.pk_fk(g, torch.zeros(4, 7, device="cuda"))[:, ee:ee + 1].contiguous()
    p = pk.pk_ik_params_default(max_iters=3, w_self=5.0)
    out = pk.pk_ik_solve(g, p, [ee], None, T, torch.zeros(4, 1, 7, device="cuda"))
    assert out[0].shape == (4, 7)
    with pytest.raises(pk.PkError) as e:
        pk.pk_ik_beam_solve(g, p, pk.pk_ik_beam_params_default(n_seeds=4), [ee], None, T,
                            torch.zeros(4, 4, 7, device="cuda"))
    assert e.value.status == pk.PK_ERR_UNSUPPORTED
    for bad in (dict(joint=[99], pairs=[]), dict(joint=[0], pairs=[[0, 0]])):
        with pytest.raises(pk.PkError):
            g.set_spheres(bad["joint"], [[0, 0, 0]], [0.1], bad["pairs"])
