"""The index-checked build (-DPK_DEBUG_BOUNDS, libpk_debug.so).

On a GPU: small workloads of every kernel family that carries checks (chain
queue with resumed records, best-seed and collision-free selection, IK-Beam,
the humanoid tree kernel, trajectories) run once against each library in a
subprocess; the checked build records no failure and returns the default
build's results bit for bit.  The status path itself is exercised by a
kernel whose one check fails without addressing anything with its index.
On the CPU: the default build reports the checks as absent and the code's
fields decode as documented."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2505_03728_gb300 import build, pk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(code_or_script, debug, *args, timeout=600):
    env = dict(os.environ, PK_DEBUG_BOUNDS="1" if debug else "0")
    env["PYTHONPATH"] = ROOT + (os.pathsep + env["PYTHONPATH"] if env.get("PYTHONPATH") else "")
    cmd = [sys.executable] + ([code_or_script] if code_or_script.endswith(".py") else ["-c", code_or_script])
    r = subprocess.run(cmd + list(args), cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return r.stdout


def test_default_build_has_no_checks():
    build.build()
    assert not pk.pk_debug_bounds_enabled()
    with pytest.raises(pk.PkError):
        pk.pk_debug_bounds_take()


def test_code_fields_decode():
    code = (4 << 48) | (64 << 24) | 70
    assert pk.pk_debug_bounds_decode(code) == (4, 64, 70)
    assert pk.pk_debug_bounds_decode((9 << 48) | (8 << 24) | 0xFFFFFF) == (9, 8, -1)


@pytest.mark.gpu
def test_checked_build_records_nothing_and_matches(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    build.build(debug_bounds=True)
    script = os.path.join(ROOT, "tests", "debug_bounds_workloads.py")
    plain, checked = str(tmp_path / "plain.npz"), str(tmp_path / "checked.npz")
    _run(script, False, plain)
    _run(script, True, checked)
    a, b = np.load(plain), np.load(checked)
    assert int(a["checked"]) == 0 and int(b["checked"]) == 1
    bounds = [k for k in b.files if k.startswith("bounds_")]
    assert len(bounds) == 6
    for k in bounds:
        assert int(b[k]) == 0, (k, pk.pk_debug_bounds_decode(int(b[k])))
    outs = [k for k in a.files if k != "checked"]
    assert len(outs) >= 20
    for k in outs:
        np.testing.assert_array_equal(b[k], a[k], err_msg=k)


@pytest.mark.gpu
def test_status_path_records_site_bound_and_index():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build(debug_bounds=True)
    code = (
        "from paper_2505_03728_gb300 import pk\n"
        "assert pk.pk_debug_bounds_enabled()\n"
        "assert pk.pk_debug_bounds_take() == 0\n"
        "pk.pk_debug_bounds_selftest(5)\n"
        "print(pk.pk_debug_bounds_decode(pk.pk_debug_bounds_take()))\n"
        "print(pk.pk_debug_bounds_take())\n"
        "pk.pk_debug_bounds_selftest(0)\n"
        "pk.pk_debug_bounds_selftest(7)\n"  # the first failure is the one kept
        "print(pk.pk_debug_bounds_decode(pk.pk_debug_bounds_take()))\n")
    lines = _run(code, True).strip().splitlines()
    assert lines[-3:] == ["(15, 5, 5)", "0", "(15, 0, 0)"]
