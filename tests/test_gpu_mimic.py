"""Mimic joints on the GPU (Sec. III-B): the 24-joint hand with the distal joint
of every finger following the joint before it (19 variables), on the
warp-per-problem path, against the FP64 oracle (itself pinned by expansion to
the plain robot in test_oracle_mimic.py)."""
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


def setup(B, S, kinds_name="position", seed=0):
    spec, tips = synth.hand_mimic_robot()
    g, o = pk.Robot.from_spec(spec), oracle.Robot.from_dict(spec)
    assert g.n_dof == o.n_dof == 19
    links = list(tips)
    kinds = [pk.PK_TARGET_POSITION] * 5 if kinds_name == "position" else [0, 1, 0, 1, 0]
    qt = synth.uniform_q(900 + seed, B, o.dof_lower, o.dof_upper)
    T = oracle.fk(o, qt)[:, links]
    sd = synth.uniform_q(910 + seed, (B, S), o.dof_lower, o.dof_upper)
    return spec, g, o, links, kinds, T, sd


def test_mimic_fk_matches_oracle():
    spec, g, o, links, kinds, T, sd = setup(64, 1)
    q = sd[:, 0]
    Tg = pk.pk_fk(g, dev(q)).cpu().numpy()
    np.testing.assert_allclose(Tg, oracle.fk(o, q), atol=2e-5)


@pytest.mark.parametrize("kinds_name", ["position", "mixed"])
def test_mimic_iterates_match_oracle(kinds_name):
    spec, g, o, links, kinds, T, sd = setup(97, 1, kinds_name)
    tg = oracle.Targets(links, kinds)
    ref = oracle.ik_solve(o, oparams(pk.pk_ik_params_default(max_iters=5, early_exit=0)), tg, T, sd, n_trace=5)
    tie = ref["margin"] <= 1e-5
    for k in range(1, 6):
        p = pk.pk_ik_params_default(max_iters=k, early_exit=0)
        q = pk.pk_ik_solve(g, p, links, kinds, dev(T), dev(sd))[0].cpu().numpy().astype(np.float64)
        qr = ref["trace"][:, k - 1]
        rel = (np.abs(q - qr) / np.maximum(1.0, np.abs(qr))).max(axis=1)
        assert np.all(rel[~tie] <= 1e-4), (kinds_name, k, np.sort(rel)[-4:])
    assert tie.sum() <= 5


def test_mimic_multistart_against_oracle():
    spec, g, o, links, kinds, T, sd = setup(256, 8, seed=1)
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=1)
    q, err, iters, status = [x.cpu().numpy() for x in pk.pk_ik_solve(g, p, links, kinds, dev(T), dev(sd))]
    tg = oracle.Targets(links, kinds)
    ref = oracle.ik_solve(o, oparams(p), tg, T, sd)
    ok, ok_ref = status == 0, ref["status"] == 0
    print(f"mimic hand: success GPU {ok.mean():.3f} oracle {ok_ref.mean():.3f}")
    assert ok.mean() >= 0.5 and abs(ok.mean() - ok_ref.mean()) <= 0.05
    for b in np.nonzero(ok)[0]:
        pe, re = oracle.ik_errors(o, tg, T[b], q[b].astype(np.float64))
        assert pe <= 1e-3 * (1 + 1e-3)


def test_mimic_argument_checks():
    spec, tips = synth.hand_mimic_robot()
    g = pk.Robot.from_spec(spec)
    mimic = np.asarray(spec["mimic"])
    j = int(np.nonzero(mimic >= 0)[0][0])
    src = int(mimic[j])
    fixed = int(np.nonzero(np.asarray(spec["type"]) == 0)[0][0])
    free = [i for i in range(len(mimic)) if spec["type"][i] != 0 and mimic[i] < 0 and i not in mimic]
    for args, why in (((j, free[0]), "already a mimic"), ((free[0], j), "source is a mimic"),
                      ((fixed, free[0]), "fixed joint"), ((free[0], free[0]), "self")):
        with pytest.raises(pk.PkError) as e:
            g.set_mimic(*args)
        assert e.value.status == pk.PK_ERR_INVALID_ARG, why
    # a serial chain with a mimic joint leaves the chain kernels
    chain = pk.Robot.from_spec(synth.chain_robot(100, 7))
    chain.set_mimic(6, 5, 0.5, 0.0)
    assert chain.n_dof == 6
    ee = chain.n_joints - 1
    q = torch.zeros(4, 1, 6, device="cuda")
    T = pk.pk_fk(chain, torch.zeros(4, 6, device="cuda"))[:, ee:ee + 1].contiguous()
    out = pk.pk_ik_solve(chain, pk.pk_ik_params_default(max_iters=3), [ee], None, T, q)
    assert out[0].shape == (4, 6)
    with pytest.raises(pk.PkError) as e:
        pk.pk_ik_residual(chain, pk.pk_ik_params_default(), [ee], None, T, torch.zeros(4, 6, device="cuda"))
    assert e.value.status == pk.PK_ERR_UNSUPPORTED


def test_seed_network_on_a_mimic_hand():
    spec, g, o, links, kinds, T, sd = setup(512, 1)
    net = pk.SeedNet(g, links, K=4, width=256, depth=2, seed=3)
    pk.pk_seednet_train(net, pk.pk_train_params_default(epochs=1, steps_per_epoch=50, batch=1024))
    s = pk.pk_seednet_infer(net, dev(T)).cpu().numpy()
    assert s.shape == (512, 4, 19)
    assert np.all(s >= o.dof_lower - 1e-5) and np.all(s <= o.dof_upper + 1e-5)
