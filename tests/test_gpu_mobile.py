"""Mobile-base IK on the GPU (Sec. V-B): the 7-DoF chain on an SE(2) base
(prismatic x, prismatic y, revolute z ahead of the arm; ten variables, the
warp-per-problem path) against the FP64 oracle, and the paper's experiment:
reachable poses shifted in the plane, solved with a fixed and with a mobile
base at 5 mm / 0.05 rad."""
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


def oparams(p):
    return oracle.IkParams(w_pos=p.w_pos, w_rot=p.w_rot, w_limit=p.w_limit, w_rest=p.w_rest, lambda0=p.lambda0,
                           lambda_min=p.lambda_min, lambda_max=p.lambda_max, nu=p.nu, tol_pos=p.tol_pos,
                           tol_rot=p.tol_rot, max_iters=p.max_iters, early_exit=p.early_exit)


def setup(B, S):
    cfg = dict(synth.MOBILE, batch=B, n_seeds=S)
    arm, mob, qt, shift, sd = synth.mobile_workload(cfg)
    oa, om = oracle.Robot.from_dict(arm), oracle.Robot.from_dict(mob)
    ee = oa.n_joints - 1
    T = oracle.fk(oa, qt)[:, ee].copy()
    T[:, 3] += shift[:, 0]
    T[:, 7] += shift[:, 1]
    seeds_m = np.concatenate([np.zeros(sd.shape[:2] + (3,)), sd], axis=2)
    return arm, mob, oa, om, ee, T[:, None], sd, seeds_m


def test_mobile_iterates_match_oracle():
    arm, mob, oa, om, ee, T, sd, sm = setup(97, 1)
    g = pk.Robot.from_spec(mob)
    tg = oracle.Targets([ee + 3])
    ref = oracle.ik_solve(om, oparams(pk.pk_ik_params_default(max_iters=5, early_exit=0)), tg, T, sm, n_trace=5)
    tie = ref["margin"] <= 1e-5
    for k in range(1, 6):
        p = pk.pk_ik_params_default(max_iters=k, early_exit=0)
        q = pk.pk_ik_solve(g, p, [ee + 3], None, dev(T), dev(sm))[0].cpu().numpy().astype(np.float64)
        qr = ref["trace"][:, k - 1]
        rel = (np.abs(q - qr) / np.maximum(1.0, np.abs(qr))).max(axis=1)
        if k <= 3:
            assert np.all(rel[~tie] <= 1e-4), (k, np.sort(rel)[-4:])
        else:
            # ten variables against six pose rows: a four-dimensional near-null
            # space held only by lambda and the 1e-6 rest weight, along which
            # FP32 rounding grows from iteration to iteration
            assert np.mean(rel[~tie] <= 1e-4) >= 0.97 and np.all(rel[~tie] <= 1e-3), (k, np.sort(rel)[-4:])
    assert tie.sum() <= 5


def test_mobile_base_solves_what_the_fixed_base_cannot():
    B = 2048
    arm, mob, oa, om, ee, T, sd, sm = setup(B, 8)
    ga, gm = pk.Robot.from_spec(arm), pk.Robot.from_spec(mob)
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=1, tol_pos=5e-3, tol_rot=0.05)
    qa, ea, _, sa = [x.cpu().numpy() for x in pk.pk_ik_solve(ga, p, [ee], None, dev(T), dev(sd))]
    qm, em, _, smob = [x.cpu().numpy() for x in pk.pk_ik_solve(gm, p, [ee + 3], None, dev(T), dev(sm))]
    fixed, mobile = (sa == 0).mean(), (smob == 0).mean()
    print(f"fixed base {fixed:.3f}, mobile base {mobile:.3f}; mean position error mobile "
          f"{ea[sa == 0, 0].mean() if fixed > 0 else float('nan'):.2e} / {em[smob == 0, 0].mean():.2e}")
    assert mobile >= 0.95 and mobile >= fixed + 0.3
    tg = oracle.Targets([ee + 3])
    for b in np.nonzero(smob == 0)[0][:300]:
        pe, re = oracle.ik_errors(om, tg, T[b], qm[b].astype(np.float64))
        assert pe <= 5e-3 * (1 + 1e-3) and re <= 0.05 * (1 + 1e-3)
    # a sample re-solved by the oracle
    idx = np.arange(0, B, 64)
    r = oracle.ik_solve(om, oparams(p), tg, T[idx], sm[idx])
    assert ((r["status"] == 0) == (smob[idx] == 0)).mean() >= 0.9
