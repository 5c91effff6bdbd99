"""GPU IK on kinematic trees with several targets (one warp per problem)
against the FP64 oracle: the 24-DoF hand with five fingertip position targets
and the 30-joint humanoid with six pose targets (and a mix of pose and
position targets).  Tolerances as for chains: LM iterates 1..5 within
1e-4 * max(1, |q|) except accept/reject near-ties; converged GPU solutions
re-checked in FP64."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_03728_gb300 import build, pk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.cpu().numpy().astype(np.float64)


def case(name, B, S, seed=0):
    if name == "hand":
        spec, links = synth.hand_robot(102)
        kinds = [pk.PK_TARGET_POSITION] * len(links)
    elif name == "humanoid":
        spec, links = synth.humanoid_robot(103)
        kinds = None
    else:
        spec, links = synth.humanoid_robot(103)
        kinds = [0, 1, 0, 1, 0, 0]
    o = oracle.Robot.from_dict(spec)
    g = pk.Robot.from_spec(spec)
    qt = synth.uniform_q(700 + seed, B, o.dof_lower, o.dof_upper)
    targets = oracle.fk(o, qt)[:, list(links)]
    seeds = synth.uniform_q(800 + seed, (B, S), o.dof_lower, o.dof_upper)
    return o, g, list(links), kinds, targets, seeds


def oparams(p):
    return oracle.IkParams(w_pos=p.w_pos, w_rot=p.w_rot, w_limit=p.w_limit, w_rest=p.w_rest, lambda0=p.lambda0,
                           lambda_min=p.lambda_min, lambda_max=p.lambda_max, nu=p.nu, tol_pos=p.tol_pos,
                           tol_rot=p.tol_rot, max_iters=p.max_iters, early_exit=p.early_exit)


@pytest.mark.parametrize("name", ["hand", "humanoid", "humanoid_mixed"])
def test_first_five_iterates_match_oracle(name):
    o, g, links, kinds, targets, seeds = case(name, 97, 1)
    ref = oracle.ik_solve(o, oparams(pk.pk_ik_params_default(max_iters=5, early_exit=0)),
                          oracle.Targets(links, kinds), targets, seeds, n_trace=5)
    tie = ref["margin"] <= 1e-5
    worst = 0.0
    for k in range(1, 6):
        p = pk.pk_ik_params_default(max_iters=k, early_exit=0)
        q, err, iters, status = [host(x) for x in pk.pk_ik_solve(g, p, links, kinds, dev(targets), dev(seeds))]
        assert np.all(iters == k)
        qr = ref["trace"][:, k - 1]
        rel = (np.abs(q - qr) / np.maximum(1.0, np.abs(qr))).max(axis=1)
        worst = max(worst, rel[~tie].max())
        assert np.all(rel[~tie] <= 1e-4), (name, k, np.sort(rel)[-4:])
    assert tie.sum() <= 5
    print(f"{name}: worst iterate error {worst:.2e}, near-ties {int(tie.sum())}/97")


@pytest.mark.parametrize("name", ["hand", "humanoid"])
def test_multistart_against_oracle(name):
    o, g, links, kinds, targets, seeds = case(name, 300, 8, seed=1)
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=1)
    q, err, iters, status = [host(x) for x in pk.pk_ik_solve(g, p, links, kinds, dev(targets), dev(seeds))]
    ref = oracle.ik_solve(o, oparams(p), oracle.Targets(links, kinds), targets, seeds)
    ok, ok_ref = status == 0, ref["status"] == 0
    print(f"{name}: success GPU {ok.mean():.3f} oracle {ok_ref.mean():.3f}")
    assert abs(ok.mean() - ok_ref.mean()) <= 0.05
    tg = oracle.Targets(links, kinds)
    for b in np.nonzero(ok)[0]:
        pe, re = oracle.ik_errors(o, tg, targets[b], q[b])
        assert pe <= 1e-3 * (1 + 1e-3) and re <= np.deg2rad(0.5) * (1 + 1e-3)
