"""The C-ABI library loads, exports every function include/pk.h declares, and
rejects malformed arguments on the host (no GPU needed: argument checks run
before any CUDA call)."""
import ctypes as C

import numpy as np
import pytest

from paper_2505_03728_gb300 import build, pk, synth


@pytest.fixture(scope="module")
def L():
    build.build()
    return pk.lib()


def test_exports_every_declared_function(L):
    names = pk.header_functions()
    assert "pk_ik_solve" in names and "pk_robot_create" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_params_default(L):
    p = pk.pk_ik_params_default()
    assert p.w_pos == 1.0 and p.w_rot == 0.5 and p.w_limit == 10.0
    assert abs(p.w_rest - 1e-3) < 1e-9 and abs(p.lambda0 - 1e-2) < 1e-9 and p.nu == 2.0
    assert abs(p.tol_rot - np.deg2rad(0.5)) < 1e-7 and abs(p.tol_pos - 1e-3) < 1e-9
    assert p.max_iters == 50 and p.early_exit == 1 and p.cancel_siblings == 0 and p.reserved == 0


def _create(spec, **mod):
    d = {k: np.array(v, copy=True) for k, v in spec.items() if k != "name"}
    d.update(mod)
    n = len(d["parent"])
    h = C.c_void_p()
    f32 = lambda a: np.ascontiguousarray(a, np.float32)
    i32 = lambda a: np.ascontiguousarray(a, np.int32)
    arrs = [i32(d["parent"]), i32(d["type"]), f32(d["axis"]), f32(d["origin"]), f32(d["lower"]),
            f32(d["upper"])]
    st = pk.lib().pk_robot_create(n, arrs[0].ctypes.data_as(pk._i32p), arrs[1].ctypes.data_as(pk._i32p),
                                  arrs[2].ctypes.data_as(pk._f32p), arrs[3].ctypes.data_as(pk._f32p),
                                  arrs[4].ctypes.data_as(pk._f32p), arrs[5].ctypes.data_as(pk._f32p),
                                  None, C.byref(h))
    return st, h


@pytest.mark.parametrize("case", ["parent_cycle", "parent_range", "bad_type", "zero_axis",
                                  "bad_limits", "nan_origin", "non_rigid_origin"])
def test_robot_create_rejects_malformed_trees(L, case):
    spec = synth.chain_robot(100, 7)
    mod = {}
    if case == "parent_cycle":
        p = spec["parent"].copy(); p[3] = 5; mod["parent"] = p
    elif case == "parent_range":
        p = spec["parent"].copy(); p[0] = -2; mod["parent"] = p
    elif case == "bad_type":
        t = spec["type"].copy(); t[2] = 7; mod["type"] = t
    elif case == "zero_axis":
        a = spec["axis"].copy(); a[1] = 0; mod["axis"] = a
    elif case == "bad_limits":
        lo = spec["lower"].copy(); lo[0] = 5.0; mod["lower"] = lo
    elif case == "nan_origin":
        o = spec["origin"].copy(); o[2, 3] = np.nan; mod["origin"] = o
    elif case == "non_rigid_origin":
        o = spec["origin"].copy(); o[2, 0] = 2.0; mod["origin"] = o
    st, h = _create(spec, **mod)
    assert st == pk.PK_ERR_INVALID_ARG
    assert not h.value
    assert len(pk.pk_last_error()) > 0


def test_null_arguments(L):
    assert L.pk_robot_create(3, None, None, None, None, None, None, None, None) == pk.PK_ERR_INVALID_ARG
    assert L.pk_fk(None, 1, None, None, None) == pk.PK_ERR_INVALID_ARG
    assert L.pk_ik_solve(None, None, 1, None, None, 1, 1, None, None, None, None, None, None, None, 0,
                         None) == pk.PK_ERR_INVALID_ARG
    assert L.pk_ik_workspace_bytes(None, 1, 1) == 0
    assert L.pk_ik_solve_split(None, None, 1, None, None, 1, 1, None, None, None, None, None, None, None, 0, 8, 0,
                               None, None) == pk.PK_ERR_INVALID_ARG
    assert L.pk_ik_split_workspace_bytes(None, 1, 1) == 0
    stats = (C.c_int64 * 8)()
    assert L.pk_ik_split_workspace_stats(None, stats) == pk.PK_ERR_INVALID_ARG
    assert L.pk_seednet_save(None, b"x.pksn") == pk.PK_ERR_INVALID_ARG
    assert L.pk_seednet_load(None, b"x.pksn") == pk.PK_ERR_INVALID_ARG


def test_trajopt_interpolate_rejects_bad_sizes_on_the_host(L):
    assert L.pk_trajopt_interpolate(-1, 4, 7, None, None, None, None) == pk.PK_ERR_INVALID_ARG
    assert L.pk_trajopt_interpolate(2, 0, 7, None, None, None, None) == pk.PK_ERR_INVALID_ARG
    assert L.pk_trajopt_interpolate(2, 4, 7, None, None, None, None) == pk.PK_ERR_INVALID_ARG  # NULL buffers
    assert L.pk_trajopt_interpolate(0, 4, 7, None, None, None, None) == pk.PK_OK  # nothing to do
