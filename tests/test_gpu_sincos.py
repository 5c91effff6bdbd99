"""Sine and cosine of the joint angles (the FK kernels' own range-reduced
polynomial) against FP64, through the public FK of a single revolute joint
about z: R = [[c, -s, 0], [s, c, 0], [0, 0, 1]].  Bound: 2e-7 absolute (a few
units in the last place of an FP32 value near 1), over angles well past the
joint limits, including the quadrant boundaries."""
import numpy as np
import pytest
import torch

from paper_2505_03728_gb300 import build, pk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


def test_sin_cos_error_bound():
    origin = np.zeros((1, 12))
    origin[0, [0, 5, 10]] = 1.0
    spec = dict(parent=[-1], type=[1], axis=[[0.0, 0.0, 1.0]], origin=origin, lower=[-100.0], upper=[100.0])
    g = pk.Robot.from_spec(spec)
    q = np.concatenate([np.linspace(-12.0, 12.0, 240001), np.arange(-8, 9) * np.pi / 2,
                        np.arange(-8, 9) * np.pi / 2 + 1e-6, np.linspace(-1e-4, 1e-4, 1001)]).astype(np.float32)
    T = pk.pk_fk(g, torch.as_tensor(q[:, None], device="cuda")).cpu().numpy().reshape(-1, 12)
    qd = q.astype(np.float64)
    err_c = np.abs(T[:, 0] - np.cos(qd)).max()
    err_s = np.abs(T[:, 4] - np.sin(qd)).max()
    print(f"max abs error: cos {err_c:.2e}, sin {err_s:.2e}")
    assert err_c <= 2e-7 and err_s <= 2e-7
    np.testing.assert_allclose(T[:, 1], -T[:, 4], atol=0)
