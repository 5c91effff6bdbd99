"""Seed network on the tensor cores against the FP64 oracle.

The GPU keeps BF16 weights and BF16 activations between layers (FP32
accumulation in TMEM), the oracle computes in FP64 from the same BF16-rounded
weights and inputs.  Tolerances: forward outputs relative L2 error <= 2e-2 and
cosine >= 0.999; gradients per layer cosine >= 0.999 and relative L2 error
<= 3e-2; loss relative error <= 1e-2.
"""
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


def bf16(a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def features(T):
    """Oracle-side features of poses [B][k][12]: t then the first two columns of R."""
    T = np.asarray(T).reshape(T.shape[0], -1, 3, 4)
    f = np.concatenate([T[..., :, 3], T[..., :, 0], T[..., :, 1]], axis=-1)
    return f.reshape(T.shape[0], -1)


def _setup(B=300, seed=0, width=512, depth=4, K=8):
    spec = synth.chain_robot(100, 7)
    g = pk.Robot.from_spec(spec)
    o = oracle.Robot.from_dict(spec)
    ee = o.n_joints - 1
    net = pk.SeedNet(g, [ee], K=K, width=width, depth=depth, seed=seed)
    rng = np.random.default_rng(seed + 10)
    dims = net.dims
    params = []
    for l in range(len(dims) - 1):
        s = 1.5 / np.sqrt(dims[l])
        params += [rng.uniform(-s, s, dims[l + 1] * dims[l]), rng.uniform(-0.1, 0.1, dims[l + 1])]
    params = bf16(np.concatenate(params))
    pk.pk_seednet_set_params(net, params)
    qt = synth.uniform_q(seed + 20, B, o.dof_lower, o.dof_upper)
    T = oracle.fk(o, qt)[:, [ee]]
    return net, o, dims, params, T, qt


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _cos(a, b):
    return float(a.ravel() @ b.ravel() / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("B", [1, 300, 4096])
def test_forward_matches_oracle(B):
    net, o, dims, params, T, qt = _setup(B)
    y = pk.pk_seednet_forward(net, dev(T)).cpu().numpy()
    x = bf16(features(T))
    ref = oracle.mlp_forward(dims, params, x)
    assert _rel(y, ref) <= 2e-2, _rel(y, ref)
    assert _cos(y, ref) >= 0.999
    np.testing.assert_array_equal(pk.pk_seednet_get_params(net), params.astype(np.float32))


def test_seeds_head_maps_into_limits():
    net, o, dims, params, T, qt = _setup(200)
    seeds = pk.pk_seednet_infer(net, dev(T)).cpu().numpy()
    y = pk.pk_seednet_forward(net, dev(T)).cpu().numpy().reshape(200, 8, 7)
    lo, hi = o.dof_lower, o.dof_upper
    np.testing.assert_allclose(seeds, (lo + hi) / 2 + (hi - lo) / 2 * np.tanh(y), atol=2e-6)
    assert np.all(seeds >= lo - 1e-6) and np.all(seeds <= hi + 1e-6)


@pytest.mark.parametrize("B", [300, 2048])
def test_loss_and_gradient_match_oracle(B):
    net, o, dims, params, T, qt = _setup(B, seed=1)
    loss, grad = pk.pk_seednet_loss_grad(net, dev(T), dev(qt))
    x = bf16(features(T))
    ref_loss, ref_grad, _ = oracle.mlp_loss_grad(dims, params, x, qt, 8, o.dof_lower, o.dof_upper, mu=0.01)
    assert abs(loss - ref_loss) <= 1e-2 * ref_loss
    off = 0
    for l in range(len(dims) - 1):
        for size in (dims[l + 1] * dims[l], dims[l + 1]):
            a, b = grad[off:off + size], ref_grad[off:off + size]
            off += size
            assert _cos(a, b) >= 0.999, (l, size, _cos(a, b))
            assert _rel(a, b) <= 3e-2, (l, size, _rel(a, b))


def test_adamw_step_matches_oracle():
    net, o, dims, params, T, qt = _setup(512, seed=2)
    tp = pk.pk_train_params_default(weight_decay=1e-4)
    lr = 1e-3
    x = bf16(features(T))
    _, ref_grad, _ = oracle.mlp_loss_grad(dims, params, x, qt, 8, o.dof_lower, o.dof_upper, mu=tp.mu)
    pk.pk_seednet_train_step(net, tp, dev(T), dev(qt), lr)
    after = pk.pk_seednet_get_params(net).astype(np.float64)
    p = params.copy()
    m, v = np.zeros_like(p), np.zeros_like(p)
    oracle.adamw(p, ref_grad, m, v, lr, tp.beta1, tp.beta2, tp.eps, tp.weight_decay, 1)
    # the first AdamW step moves each parameter by about lr * sign(g): compare where the
    # gradient is not negligible
    big = np.abs(ref_grad) > 1e-3 * np.abs(ref_grad).max()
    close = np.abs(after - p) <= 1e-6 + 1e-2 * lr
    assert close[big].mean() >= 0.99


def test_training_reduces_loss():
    spec = synth.chain_robot(100, 7)
    g = pk.Robot.from_spec(spec)
    net = pk.SeedNet(g, [g.n_joints - 1], K=8, width=512, depth=4, seed=3)
    tp = pk.pk_train_params_default(epochs=3, steps_per_epoch=60, batch=4096)
    losses = pk.pk_seednet_train(net, tp)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.8 * losses[0], losses
