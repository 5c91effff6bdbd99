"""Pins for the FP64 seed-network oracle: forward, min-over-K loss and its
gradient against PyTorch float64 autograd on the CPU (an independent
implementation of the same definition), central finite differences, and the
AdamW step against torch.optim.AdamW."""
import numpy as np
import pytest
import torch

import oracle

DIMS = [9, 24, 24, 3 * 4]  # small network: K = 3 proposals of n = 4 joints


def _setup(seed=0, M=17):
    rng = np.random.default_rng(seed)
    params = rng.normal(0, 0.4, oracle.mlp_n_params(DIMS))
    x = rng.normal(0, 1, (M, DIMS[0]))
    q_star = rng.uniform(-2, 2, (M, 4))
    lo, hi = np.full(4, -2.8), np.full(4, 2.8)
    return params, x, q_star, lo, hi


def _torch_model(params):
    out, off = [], 0
    for l in range(len(DIMS) - 1):
        W = torch.tensor(params[off:off + DIMS[l + 1] * DIMS[l]].reshape(DIMS[l + 1], DIMS[l]),
                         dtype=torch.float64, requires_grad=True)
        off += DIMS[l + 1] * DIMS[l]
        b = torch.tensor(params[off:off + DIMS[l + 1]], dtype=torch.float64, requires_grad=True)
        off += DIMS[l + 1]
        out += [W, b]
    return out


def _torch_loss(tp, x, q_star, lo, hi, K=3, mu=0.01):
    a = torch.tensor(x)
    L = len(DIMS) - 1
    for l in range(L):
        a = torch.nn.functional.linear(a, tp[2 * l], tp[2 * l + 1])
        if l + 1 < L:
            a = torch.nn.functional.silu(a)
    y = a.reshape(x.shape[0], K, -1)
    lo_t, hi_t = torch.tensor(lo), torch.tensor(hi)
    q = (lo_t + hi_t) / 2 + (hi_t - lo_t) / 2 * torch.tanh(y)
    e = ((q - torch.tensor(q_star)[:, None, :]) ** 2).sum(-1)
    return (e.min(dim=1).values + mu * e.mean(dim=1)).mean(), a, q


def test_forward_matches_torch():
    params, x, q_star, lo, hi = _setup()
    y = oracle.mlp_forward(DIMS, params, x)
    _, a, _ = _torch_loss(_torch_model(params), x, q_star, lo, hi)
    np.testing.assert_allclose(y, a.detach().numpy(), rtol=1e-12, atol=1e-12)


def test_loss_and_gradient_match_torch_autograd():
    params, x, q_star, lo, hi = _setup(1)
    loss, grad, q = oracle.mlp_loss_grad(DIMS, params, x, q_star, 3, lo, hi)
    tp = _torch_model(params)
    tl, _, tq = _torch_loss(tp, x, q_star, lo, hi)
    tl.backward()
    tg = np.concatenate([t.grad.numpy().ravel() for t in tp])
    assert abs(loss - tl.item()) <= 1e-12 * max(1, abs(loss))
    np.testing.assert_allclose(q, tq.detach().numpy(), atol=1e-12)
    np.testing.assert_allclose(grad, tg, rtol=1e-9, atol=1e-12)


def test_gradient_matches_central_fd():
    params, x, q_star, lo, hi = _setup(2, M=5)
    _, grad, _ = oracle.mlp_loss_grad(DIMS, params, x, q_star, 3, lo, hi)
    rng = np.random.default_rng(3)
    h = 1e-6
    for i in rng.choice(params.size, 40, replace=False):
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (oracle.mlp_loss_grad(DIMS, p1, x, q_star, 3, lo, hi)[0]
              - oracle.mlp_loss_grad(DIMS, p2, x, q_star, 3, lo, hi)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])), i


def test_adamw_matches_torch():
    rng = np.random.default_rng(4)
    p = rng.normal(size=50)
    tparam = torch.tensor(p.copy(), requires_grad=True)
    opt = torch.optim.AdamW([tparam], lr=1e-2, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-2)
    m, v = np.zeros(50), np.zeros(50)
    for step in range(1, 6):
        g = rng.normal(size=50)
        oracle.adamw(p, g, m, v, 1e-2, 0.9, 0.999, 1e-8, 1e-2, step)
        tparam.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(p, tparam.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_round_bf16_matches_torch_bfloat16():
    """BF16 rounding (8 significant bits, ties to even) against PyTorch's
    bfloat16 cast, on float32 values (the cast rounds from float32) including
    exact ties."""
    rng = np.random.default_rng(7)
    x = rng.standard_normal(20000).astype(np.float32).astype(np.float64) * 10.0 ** rng.integers(-6, 6, 20000)
    x = x.astype(np.float32).astype(np.float64)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -3 * (1 + 5 * 2 ** -8), 0.0, -0.0])
    for v in (x, ties):
        ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
        np.testing.assert_array_equal(oracle.round_bf16(v), ref)
    np.testing.assert_array_equal(oracle.round_bf16(ties[:4]), [1.0, 1 + 2 ** -6, -1.0, 2 ** -3 * (1 + 4 * 2 ** -8)])


def test_forward_bf16_matches_torch_with_bf16_activations():
    """The forward pass at the network's precision: the same layers with every
    hidden SiLU output cast to bfloat16 by PyTorch, and the output layer's
    magnitude scale sum |W||a| + |b|."""
    params, x, q_star, lo, hi = _setup(seed=4)
    y, scale = oracle.mlp_forward_bf16(DIMS, params, x)
    tp = _torch_model(params)
    a = torch.tensor(x)
    L = len(DIMS) - 1
    for l in range(L):
        z = torch.nn.functional.linear(a, tp[2 * l], tp[2 * l + 1])
        if l + 1 < L:
            a = torch.nn.functional.silu(z).to(torch.float32).to(torch.bfloat16).to(torch.float64)
        else:
            mag = torch.nn.functional.linear(a.abs(), tp[2 * l].abs(), tp[2 * l + 1].abs())
            a = z
    np.testing.assert_allclose(y, a.detach().numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(scale, mag.detach().numpy(), rtol=1e-12)
    assert np.abs(y - oracle.mlp_forward(DIMS, params, x)).max() > 0  # the rounding does act
