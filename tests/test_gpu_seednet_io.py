"""pk_seednet_save / pk_seednet_load: a saved network loads into another
network of the same shape with identical parameters and seeds; files of
another shape, truncated files and missing paths are rejected with the
network left unchanged."""
import numpy as np
import pytest
import torch

from paper_2505_03728_gb300 import build, pk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    pk.lib()


def net_pair(width=256, depth=2, K=4):
    g = pk.Robot.from_spec(synth.chain_robot(100, 7))
    ee = g.n_joints - 1
    return g, ee, pk.SeedNet(g, [ee], K=K, width=width, depth=depth, seed=1), \
        pk.SeedNet(g, [ee], K=K, width=width, depth=depth, seed=2)


def test_round_trip_gives_identical_parameters_and_seeds(tmp_path):
    g, ee, a, b = net_pair()
    pa = pk.pk_seednet_get_params(a)
    assert not np.array_equal(pa, pk.pk_seednet_get_params(b))
    path = str(tmp_path / "net.pksn")
    pk.pk_seednet_save(a, path)
    pk.pk_seednet_load(b, path)
    np.testing.assert_array_equal(pk.pk_seednet_get_params(b), pa)
    q = torch.as_tensor(synth.uniform_q(3, 500, np.full(7, -2.8), np.full(7, 2.8)), dtype=torch.float32,
                        device="cuda")
    T = pk.pk_fk(g, q)[:, ee:ee + 1].contiguous()
    assert torch.equal(pk.pk_seednet_infer(a, T), pk.pk_seednet_infer(b, T))


def test_wrong_shape_truncated_and_missing_files_are_rejected(tmp_path):
    g, ee, a, b = net_pair()
    path = str(tmp_path / "net.pksn")
    pk.pk_seednet_save(a, path)
    before = pk.pk_seednet_get_params(b)
    wide = pk.SeedNet(g, [ee], K=4, width=512, depth=2, seed=3)
    with pytest.raises(pk.PkError):
        pk.pk_seednet_load(wide, path)
    data = open(path, "rb").read()
    short = str(tmp_path / "short.pksn")
    open(short, "wb").write(data[:len(data) - 8])
    with pytest.raises(pk.PkError):
        pk.pk_seednet_load(b, short)
    junk = str(tmp_path / "junk.pksn")
    open(junk, "wb").write(b"not a network" * 8)
    with pytest.raises(pk.PkError):
        pk.pk_seednet_load(b, junk)
    with pytest.raises(pk.PkError):
        pk.pk_seednet_load(b, str(tmp_path / "missing.pksn"))
    np.testing.assert_array_equal(pk.pk_seednet_get_params(b), before)
