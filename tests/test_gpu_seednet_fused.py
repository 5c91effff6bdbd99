"""Whole-network seed inference (one persistent tcgen05 kernel: features,
hidden layers with the activations kept in tensor memory as the MMA's A
operand, joint-limit head) against the layer-by-layer GEMM path and the FP64
oracle.

Both GPU paths run the same MMA shapes in the same K order and the same
epilogue arithmetic, so their seeds agree to FP32 rounding of the head
(bitwise on almost every element); against the oracle the tolerances of
test_gpu_seednet.py apply (relative L2 <= 2e-2, cosine >= 0.999 on the
pre-tanh outputs, here compared after the head).
"""
import os

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
    T = np.asarray(T).reshape(T.shape[0], -1, 3, 4)
    f = np.concatenate([T[..., :, 3], T[..., :, 0], T[..., :, 1]], axis=-1)
    return f.reshape(T.shape[0], -1)


ROBOTS = {
    "chain7": lambda: (synth.chain_robot(100, 7), None),
    "hand24": lambda: synth.hand_robot(102),
    "humanoid30": lambda: synth.humanoid_robot(103),
}


def make(robot, K, width, depth, B, seed=0):
    spec, tips = ROBOTS[robot]()
    g, o = pk.Robot.from_spec(spec), oracle.Robot.from_dict(spec)
    links = [o.n_joints - 1] if tips is None else list(tips)
    net = pk.SeedNet(g, links, K=K, width=width, depth=depth, seed=seed)
    rng = np.random.default_rng(seed + 10)
    dims = net.dims
    params = []
    for l in range(len(dims) - 1):
        s = 1.5 / np.sqrt(dims[l])
        params += [rng.uniform(-s, s, dims[l + 1] * dims[l]), rng.uniform(-0.1, 0.1, dims[l + 1])]
    params = bf16(np.concatenate(params))
    pk.pk_seednet_set_params(net, params)
    qt = synth.uniform_q(seed + 20, B, o.dof_lower, o.dof_upper)
    T = oracle.fk(o, qt)[:, links]
    return net, o, dims, params, T


def infer(net, T, fused):
    old = os.environ.get("PK_SEEDNET_FUSED")
    os.environ["PK_SEEDNET_FUSED"] = "1" if fused else "0"
    try:
        return pk.pk_seednet_infer(net, dev(T)).cpu().numpy()
    finally:
        if old is None:
            del os.environ["PK_SEEDNET_FUSED"]
        else:
            os.environ["PK_SEEDNET_FUSED"] = old


CASES = [  # robot, K, width, depth, batch
    ("chain7", 8, 512, 4, 1),
    ("chain7", 8, 512, 4, 128),
    ("chain7", 8, 512, 4, 300),
    ("chain7", 8, 512, 4, 20011),
    ("chain7", 8, 512, 4, 65536),  # the benchmark's batch and launch configuration
    ("chain7", 4, 256, 2, 1000),
    ("chain7", 8, 256, 1, 257),
    ("hand24", 8, 512, 3, 700),
    ("humanoid30", 8, 512, 4, 999),
]


@pytest.mark.parametrize("robot,K,width,depth,B", CASES)
def test_fused_matches_layerwise(robot, K, width, depth, B):
    net, o, dims, params, T = make(robot, K, width, depth, B)
    a = infer(net, T, True)
    b = infer(net, T, False)
    assert a.shape == b.shape == (B, K, o.n_dof)
    same = np.mean(a == b)
    print(f"{robot} K={K} w={width} d={depth} B={B}: bitwise equal {same:.4f}, max diff {np.abs(a - b).max():.2e}")
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-5)
    assert same >= 0.99


@pytest.mark.parametrize("robot,K,width,depth,B", [("chain7", 8, 512, 4, 300), ("chain7", 4, 256, 2, 1000),
                                                   ("humanoid30", 8, 512, 4, 999)])
def test_fused_matches_oracle(robot, K, width, depth, B):
    net, o, dims, params, T = make(robot, K, width, depth, B)
    q = infer(net, T, True).astype(np.float64)
    y = oracle.mlp_forward(dims, params, bf16(features(T)))[:, :K * o.n_dof].reshape(B, K, o.n_dof)
    lo, hi = o.dof_lower, o.dof_upper
    ref = (lo + hi) / 2 + (hi - lo) / 2 * np.tanh(y)
    # compare in the pre-image of the head, where the oracle's tolerance is stated
    z = np.arctanh(np.clip((2 * q - (lo + hi)) / (hi - lo), -1 + 1e-6, 1 - 1e-6))
    zr = np.arctanh(np.clip((2 * ref - (lo + hi)) / (hi - lo), -1 + 1e-6, 1 - 1e-6))
    rel = np.linalg.norm(z - zr) / np.linalg.norm(zr)
    cos = float(z.ravel() @ zr.ravel() / (np.linalg.norm(z) * np.linalg.norm(zr)))
    assert rel <= 2e-2 and cos >= 0.999, (rel, cos)
    assert np.all(q >= lo - 1e-6) and np.all(q <= hi + 1e-6)


def test_fused_inference_graph_replay_and_stream():
    net, o, dims, params, T = make("chain7", 8, 512, 4, 4096)
    x = dev(T)
    out = torch.empty(4096, 8, 7, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pk.pk_seednet_infer(net, x, out, stream=s)
    s.synchronize()
    ref = out.clone()
    g = torch.cuda.CUDAGraph()
    out.zero_()
    with torch.cuda.graph(g, stream=s):
        pk.pk_seednet_infer(net, x, out, stream=s)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_check_reports_no_device_failure_after_inference():
    net, o, dims, params, T = make("chain7", 8, 512, 4, 3000)
    infer(net, T, True)
    pk.pk_seednet_check(net)  # raises PkError on a recorded pipeline timeout
    infer(net, T, False)
    pk.pk_seednet_check(net)


def test_shapes_outside_the_fused_kernel_use_the_gemms():
    # 16 seeds x 30 joints = 480 head outputs (> 256) and width 1024: the
    # layer-by-layer GEMMs serve both, with or without PK_SEEDNET_FUSED
    for robot, K, width, depth in (("humanoid30", 16, 512, 2), ("chain7", 8, 1024, 2)):
        net, o, dims, params, T = make(robot, K, width, depth, 300)
        a = infer(net, T, True)
        b = infer(net, T, False)
        assert a.shape == (300, K, o.n_dof)
        np.testing.assert_array_equal(a, b)
        pk.pk_seednet_check(net)
