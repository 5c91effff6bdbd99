"""What the trained seed network gains over random multi-start seeds.

A network trained on the GPU (FK samples of uniform random configurations)
proposes K = 8 seeds for held-out targets; the same LM settings refine them
and refine 8 uniform random seeds.  The learned seeds must solve at least as
many targets and need fewer LM iterations to reach the tolerance."""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_03728_gb300 import build, pk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    spec = synth.chain_robot(100, 7)
    g = pk.Robot.from_spec(spec)
    ee = g.n_joints - 1
    net = pk.SeedNet(g, [ee], K=8, width=512, depth=4, seed=7)
    tp = pk.pk_train_params_default(epochs=4, steps_per_epoch=600, batch=8192, seed=500)
    losses = pk.pk_seednet_train(net, tp)
    return spec, g, ee, net, losses


def test_learned_seeds_beat_random_seeds(trained):
    spec, g, ee, net, losses = trained
    assert losses[-1] < losses[0]
    B = 8192
    qt = synth.uniform_q(501, B, spec.dof_lower, spec.dof_upper)  # held-out targets
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    targets = pk.pk_fk(g, dev(qt))[:, ee:ee + 1].contiguous()
    learned = pk.pk_seednet_infer(net, targets)
    rand = dev(synth.uniform_q(502, (B, 8), spec.dof_lower, spec.dof_upper))
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    ql, el, il, sl = [x.cpu().numpy() for x in pk.pk_ik_solve(g, p, [ee], None, targets, learned)]
    qr, er, ir, sr = [x.cpu().numpy() for x in pk.pk_ik_solve(g, p, [ee], None, targets, rand)]
    ok_l, ok_r = sl == 0, sr == 0
    print(f"success learned {ok_l.mean():.4f} random {ok_r.mean():.4f}; "
          f"mean iterations of solved targets learned {il[ok_l].mean():.2f} random {ir[ok_r].mean():.2f}")
    assert ok_l.mean() >= ok_r.mean()
    assert il[ok_l].mean() < ir[ok_r].mean()
    # the learned path's solutions are valid in FP64
    o = oracle.Robot.from_dict(spec)
    tg = oracle.Targets([ee])
    T = targets.cpu().numpy()
    for b in np.nonzero(ok_l)[0][:500]:
        pe, re = oracle.ik_errors(o, tg, T[b], ql[b])
        assert pe <= 1e-3 * (1 + 1e-3) and re <= np.deg2rad(0.5) * (1 + 1e-3)


def test_refined_pool_labels_are_ik_solutions(trained):
    """An LM refinement round: every pool label reaches its pool target in FP64
    (LM solutions within the success thresholds, the rest exact preimages)."""
    spec, g, ee, net, losses = trained
    n = 4096
    conv = pk.pk_seednet_refine(net, n, max_iters=20, seed=777)
    T, q = pk.pk_seednet_pool(net)
    assert T.shape == (n, 1, 12) and q.shape == (n, 7)
    assert conv >= 0.9 * n
    o = oracle.Robot.from_dict(spec)
    tg = oracle.Targets([ee])
    Th, qh = T.cpu().numpy().astype(np.float64), q.cpu().numpy().astype(np.float64)
    for b in range(0, n, 4):
        pe, re = oracle.ik_errors(o, tg, Th[b], qh[b])
        assert pe <= 1e-3 * (1 + 1e-3) and re <= np.deg2rad(0.5) * (1 + 1e-3)


def test_humanoid_learned_seeds_beat_random_seeds():
    """The 30-joint humanoid with six pose targets (54 input features, 8 x 30
    outputs): learned proposals against uniform random seeds, same LM."""
    spec, ends = synth.humanoid_robot(103)
    links = list(ends)
    g = pk.Robot.from_spec(spec)
    net = pk.SeedNet(g, links, K=8, width=512, depth=4, seed=5)
    tp = pk.pk_train_params_default(epochs=4, steps_per_epoch=600, batch=8192, seed=510, refine_every=2,
                                    refine_n=16384)
    losses = pk.pk_seednet_train(net, tp)
    assert losses[-1] < losses[0]
    B = 2048
    qt = synth.uniform_q(511, B, spec.dof_lower, spec.dof_upper)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    targets = pk.pk_fk(g, dev(qt))[:, links].contiguous()
    p = pk.pk_ik_params_default(max_iters=50, early_exit=1, cancel_siblings=0)
    learned = pk.pk_seednet_infer(net, targets)
    rand = dev(synth.uniform_q(512, (B, 8), spec.dof_lower, spec.dof_upper))
    ql, _, il, sl = [x.cpu().numpy() for x in pk.pk_ik_solve(g, p, links, None, targets, learned)]
    _, _, ir, sr = [x.cpu().numpy() for x in pk.pk_ik_solve(g, p, links, None, targets, rand)]
    ok_l, ok_r = sl == 0, sr == 0
    print(f"humanoid success learned {ok_l.mean():.4f} random {ok_r.mean():.4f}")
    assert ok_l.mean() >= 0.5 and ok_l.mean() >= 3 * ok_r.mean()
    o = oracle.Robot.from_dict(spec)
    tg = oracle.Targets(links)
    T = targets.cpu().numpy()
    for b in np.nonzero(ok_l)[0][:200]:
        pe, re = oracle.ik_errors(o, tg, T[b], ql[b])
        assert pe <= 1e-3 * (1 + 1e-3) and re <= np.deg2rad(0.5) * (1 + 1e-3)
