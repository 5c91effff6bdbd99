"""The FLOP census (oracle/flopcount.hpp, oracle/census.py): the counting
double computes exactly what the plain oracle computes, counts closed-form
operation totals on kernels whose work is known (dense Cholesky, the
normal-equation product), treats exact-zero operands as structural, and the
benchmark's roofline constants are the census's current output."""
import ctypes as C
import importlib
import os
import sys

import numpy as np
import pytest

import oracle
from oracle import census
from paper_2505_03728_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _counts():
    out = np.zeros(2, np.int64)
    oracle.flops_lib().orf_read(out.ctypes.data_as(C.POINTER(C.c_int64)))
    return int(out[0]), int(out[1])


def _f64p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def test_counting_build_computes_the_same_values():
    spec = synth.chain_robot(100, 7)
    rb = oracle.Robot.from_dict(spec)
    ee = rb.n_joints - 1
    tg = oracle.Targets([ee])
    prm = oracle.IkParams()
    rng = np.random.default_rng(1)
    F = oracle.flops_lib()
    for _ in range(8):
        q = rng.uniform(-2.8, 2.8, 7)
        target = oracle.fk(rb, rng.uniform(-2.8, 2.8, 7))[ee]
        r0, J0 = oracle.ik_residual(rb, prm, tg, target, q)
        m = len(r0)
        r1, J1 = np.empty(m), np.empty((m, 7))
        F.or_ik_residual(C.byref(rb._c), C.byref(prm._c), C.byref(tg._c), _f64p(np.ascontiguousarray(target)),
                         _f64p(q), _f64p(r1), _f64p(J1))
        assert np.array_equal(r0, r1) and np.array_equal(J0, J1)


@pytest.mark.parametrize("n", [1, 7, 30])
def test_dense_cholesky_solve_count_is_the_closed_form(n):
    """Factor: column j costs j mul + j sub + 1 sqrt for the pivot and, for
    each of the n-1-j rows below, j mul + j sub + 1 div; each substitution
    costs i mul + i sub + 1 div per row.  A dense SPD matrix has no exact
    zeros, so the structural-zero rule skips nothing here."""
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    b = rng.standard_normal(n)
    x = np.empty(n)
    F = oracle.flops_lib()
    F.orf_reset()
    assert F.or_cholesky_solve(n, _f64p(A), _f64p(b), _f64p(x)) == 0
    got, special = _counts()
    expect = sum((2 * j + 1) * (n - j) for j in range(n)) + 2 * n * n
    assert got == expect and special == 0
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-12)


def test_normal_equation_count_and_structural_zeros():
    """g and the lower triangle of J^T J: each entry is a sum of m products,
    m multiplies and m - 1 adds (the first add is onto an exact zero).  A zero
    row of J costs nothing."""
    rng = np.random.default_rng(3)
    m, nd = 20, 7
    J = rng.standard_normal((m, nd))
    r = rng.standard_normal(m)
    A, g = np.empty((nd, nd)), np.empty(nd)
    F = oracle.flops_lib()
    F.orf_reset()
    F.or_normal_equations(m, nd, _f64p(J), _f64p(r), _f64p(A), _f64p(g))
    dense = _counts()[0]
    assert dense == (2 * m - 1) * (nd + nd * (nd + 1) // 2)
    np.testing.assert_allclose(A, J.T @ J, rtol=1e-13)
    np.testing.assert_allclose(g, J.T @ r, rtol=1e-13)
    J[6:] = 0.0  # only the six pose rows carry values
    F.orf_reset()
    F.or_normal_equations(m, nd, _f64p(J), _f64p(r), _f64p(A), _f64p(g))
    assert _counts()[0] == (2 * 6 - 1) * (nd + nd * (nd + 1) // 2)


def test_ik_unit_counts_are_positive_and_state_dependent_only_slightly():
    out = census.ik_chain7(n_targets=2, n_seeds=2)
    for k in ("eval", "build", "solve"):
        assert out[k]["flops"] > 0
        assert out[k]["max"] <= 1.1 * out[k]["min"]
    assert out["solve"]["flops"] == sum((2 * j + 1) * (7 - j) for j in range(7)) + 2 * 49 + 2 * 7


def test_bench_constants_match_the_census():
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    c = census.census()
    ik, tr, net = c["ik_chain7"], c["trajopt7_T64"], c["seednet7"]
    assert bench.FLOPS_PER_EVAL == pytest.approx(ik["eval"]["flops"], rel=1e-3)
    assert bench.FLOPS_PER_BUILD == pytest.approx(ik["build"]["flops"], rel=1e-3)
    assert bench.FLOPS_PER_SOLVE == pytest.approx(ik["solve"]["flops"], rel=1e-3)
    assert bench.TRAJ_FLOPS_PER_ITER == pytest.approx(tr["flops_per_traj_iter"], rel=1e-3)
    assert bench.TRAJ_FLOPS_PER_INIT == pytest.approx(tr["flops_per_traj_init"], rel=1e-3)
    assert bench.seednet_flops(9, 512, 4, 56, 1) == net["flops_per_target"]
