"""FP64 CPU oracle for the batched Levenberg-Marquardt kinematic optimiser.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The library product
(``paper_2505_03728_gb300``) never imports this package, and this package
never imports the product: the two share only the seeded input generators.

The arithmetic lives in plain C (``pk_oracle.c``, ``trajopt_oracle.c``,
``mlp_oracle.c``), compiled with gcc into ``oracle/_build/libpk_oracle.so``;
this module is the ctypes marshalling around it.  Each C function cites the
paper passage it follows (Sec. III-A solver, Sec. III-B variables, Sec. III-C
costs and Eq. 1).  The same C sources compiled as C++ with a counting double
(``flopcount.hpp``, ``flops_*.cpp``) give the FLOP census of ``census.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpk_oracle.so")
_SOURCES = ["pk_oracle.c", "trajopt_oracle.c", "mlp_oracle.c"]
# the same sources compiled as C++ with the counting double of flopcount.hpp
_FLOPS_PATH = os.path.join(_BUILD, "libpk_oracle_flops.so")
_FLOPS_SOURCES = ["flops_pk.cpp", "flops_traj.cpp"]
_lock = threading.Lock()
_lib = None
_flib = None

JOINT_FIXED, JOINT_REVOLUTE, JOINT_PRISMATIC = 0, 1, 2
TARGET_POSE, TARGET_POSITION = 0, 1
P_CONVERGED, P_MAX_ITERS, P_NONFINITE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction, no -march)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "pk_oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp] + srcs + [
        "-lpthread", "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    try:
        build_flops(force)
    except (OSError, subprocess.CalledProcessError) as e:  # the census alone needs g++
        print(f"oracle: FLOP census not built ({e})")
    return _LIB_PATH


def build_flops(force: bool = False) -> str:
    """Compile the FLOP census: the oracle's C sources again, as C++, with
    every double replaced by the counting type of flopcount.hpp."""
    deps = [os.path.join(_HERE, s) for s in _FLOPS_SOURCES + ["flopcount.hpp", "pk_oracle.h"] + _SOURCES[:2]]
    newest = max(os.path.getmtime(s) for s in deps)
    if not force and os.path.exists(_FLOPS_PATH) and os.path.getmtime(_FLOPS_PATH) >= newest:
        return _FLOPS_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _FLOPS_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-Wl,-Bsymbolic",
           "-Wno-class-memaccess", "-o", tmp] + [os.path.join(_HERE, s) for s in _FLOPS_SOURCES] + ["-lpthread"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _FLOPS_PATH)
    return _FLOPS_PATH


def flops_lib():
    global _flib
    with _lock:
        if _flib is None:
            build_flops()
            _flib = C.CDLL(_FLOPS_PATH)
    return _flib


_i32p = C.POINTER(C.c_int32)
_f64p = C.POINTER(C.c_double)


class _Robot(C.Structure):
    _fields_ = [("n_joints", C.c_int32), ("parent", _i32p), ("type", _i32p), ("axis", _f64p),
                ("origin", _f64p), ("lower", _f64p), ("upper", _f64p), ("mimic", _i32p),
                ("mimic_mult", _f64p), ("mimic_off", _f64p), ("n_spheres", C.c_int32), ("sph_joint", _i32p),
                ("sph_centre", _f64p), ("sph_radius", _f64p), ("n_pairs", C.c_int32), ("pairs", _i32p)]


class _IkParams(C.Structure):
    _fields_ = [("w_pos", C.c_double), ("w_rot", C.c_double), ("w_limit", C.c_double),
                ("w_rest", C.c_double), ("lambda0", C.c_double), ("lambda_min", C.c_double),
                ("lambda_max", C.c_double), ("nu", C.c_double), ("tol_pos", C.c_double),
                ("tol_rot", C.c_double), ("max_iters", C.c_int32), ("early_exit", C.c_int32),
                ("w_self", C.c_double), ("eta_self", C.c_double)]


class _TargetSpec(C.Structure):
    _fields_ = [("n_targets", C.c_int32), ("links", _i32p), ("kinds", _i32p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            L.or_n_dof.restype = C.c_int32
            L.or_n_residuals.restype = C.c_int32
            L.or_cholesky_solve.restype = C.c_int32
            L.or_ik_solve.restype = C.c_int32
            for name in ("or_traj_solve", "or_mlp_forward", "or_mlp_loss_grad", "or_traj_n_residuals",
                         "or_banded_cholesky", "or_banded_cholesky_b", "or_host_cores", "or_ik_beam"):
                if hasattr(L, name):
                    getattr(L, name).restype = C.c_int32
            L.or_lm_run.restype = C.c_int32
            for name in ("or_coll_activation", "or_traj_normal", "or_traj_lm_run"):
                getattr(L, name).restype = C.c_double
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    if a is None:
        return None
    if a.dtype == np.float64:
        return a.ctypes.data_as(_f64p)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_i32p)
    raise TypeError(a.dtype)


class Robot:
    """A kinematic tree: parent[j] < j, joint types 0/1/2, axes, origins, limits."""

    def __init__(self, parent, type, axis, origin, lower, upper, mimic=None, mimic_mult=None, mimic_off=None,
                 spheres=None):
        self.parent = _i32(parent)
        self.type = _i32(type)
        self.axis = _f64(axis).reshape(-1, 3)
        self.origin = _f64(origin).reshape(-1, 12)
        self.lower = _f64(lower)
        self.upper = _f64(upper)
        self.n_joints = int(self.parent.shape[0])
        self.mimic = None if mimic is None else _i32(mimic)
        self.mimic_mult = None if mimic is None else _f64(mimic_mult)
        self.mimic_off = None if mimic is None else _f64(mimic_off)
        # spheres: dict(joint [S], centre [S][3], radius [S], pairs [P][2]) or None
        self.sph_joint = self.sph_centre = self.sph_radius = self.pairs = None
        n_s = n_p = 0
        if spheres is not None:
            self.sph_joint = _i32(spheres["joint"])
            self.sph_centre = _f64(spheres["centre"]).reshape(-1, 3)
            self.sph_radius = _f64(spheres["radius"])
            self.pairs = _i32(spheres["pairs"]).reshape(-1, 2)
            n_s, n_p = int(self.sph_joint.shape[0]), int(self.pairs.shape[0])
        self.n_pairs = n_p
        self._c = _Robot(self.n_joints, _p(self.parent), _p(self.type), _p(self.axis),
                         _p(self.origin), _p(self.lower), _p(self.upper), _p(self.mimic), _p(self.mimic_mult),
                         _p(self.mimic_off), n_s, _p(self.sph_joint), _p(self.sph_centre), _p(self.sph_radius),
                         n_p, _p(self.pairs))
        self.n_dof = int(lib().or_n_dof(C.byref(self._c)))

    @classmethod
    def from_dict(cls, d):
        return cls(d["parent"], d["type"], d["axis"], d["origin"], d["lower"], d["upper"], d.get("mimic"),
                   d.get("mimic_mult"), d.get("mimic_off"), d.get("spheres"))

    def _own_var(self):
        own = self.type != JOINT_FIXED
        if self.mimic is not None:
            own &= self.mimic < 0
        return own

    @property
    def dof_lower(self):
        return self.lower[self._own_var()]

    @property
    def dof_upper(self):
        return self.upper[self._own_var()]


class IkParams:
    def __init__(self, w_pos=1.0, w_rot=0.5, w_limit=10.0, w_rest=1e-3, lambda0=1e-2,
                 lambda_min=1e-10, lambda_max=1e10, nu=2.0, tol_pos=1e-3,
                 tol_rot=np.deg2rad(0.5), max_iters=30, early_exit=0, w_self=0.0, eta_self=0.02):
        self._c = _IkParams(w_pos, w_rot, w_limit, w_rest, lambda0, lambda_min, lambda_max, nu,
                            tol_pos, tol_rot, max_iters, early_exit, w_self, eta_self)

    def __getattr__(self, k):
        return getattr(self.__dict__["_c"], k)


class Targets:
    def __init__(self, links, kinds=None):
        self.links = _i32(links)
        self.kinds = None if kinds is None else _i32(kinds)
        self._c = _TargetSpec(int(self.links.shape[0]), _p(self.links), _p(self.kinds))
        self.k = int(self.links.shape[0])


def fk(robot: Robot, q) -> np.ndarray:
    """All joint frames: [..., n_joints, 12] (3x4 row-major)."""
    q = _f64(q)
    flat = q.reshape(-1, robot.n_dof)
    out = np.empty((flat.shape[0], robot.n_joints, 12))
    for i in range(flat.shape[0]):
        row = np.ascontiguousarray(flat[i])
        lib().or_fk(C.byref(robot._c), _p(row), out[i].ctypes.data_as(_f64p))
    return out.reshape(q.shape[:-1] + (robot.n_joints, 12))


def se3_log(T):
    T = _f64(T)
    out = np.empty(6)
    lib().or_se3_log(_p(T), _p(out))
    return out


def se3_exp(xi):
    xi = _f64(xi)
    out = np.empty(12)
    lib().or_se3_exp(_p(xi), _p(out))
    return out


def se3_jl(xi):
    xi = _f64(xi)
    out = np.empty((6, 6))
    lib().or_se3_jl(_p(xi), out.ctypes.data_as(_f64p))
    return out


def se3_jlinv(xi):
    xi = _f64(xi)
    out = np.empty((6, 6))
    lib().or_se3_jlinv(_p(xi), out.ctypes.data_as(_f64p))
    return out


def n_residuals(robot: Robot, tg: Targets) -> int:
    return int(lib().or_n_residuals(C.byref(robot._c), C.byref(tg._c)))


def ik_residual(robot: Robot, params: IkParams, tg: Targets, targets, q, jacobian=True):
    targets = _f64(targets).reshape(tg.k, 12)
    q = _f64(q)
    m = n_residuals(robot, tg)
    r = np.empty(m)
    J = np.empty((m, robot.n_dof)) if jacobian else None
    lib().or_ik_residual(C.byref(robot._c), C.byref(params._c), C.byref(tg._c), _p(targets),
                         _p(q), _p(r), None if J is None else J.ctypes.data_as(_f64p))
    return (r, J) if jacobian else r


def ik_errors(robot: Robot, tg: Targets, targets, q):
    targets = _f64(targets).reshape(tg.k, 12)
    q = _f64(q)
    pe, re = C.c_double(), C.c_double()
    lib().or_ik_errors(C.byref(robot._c), C.byref(tg._c), _p(targets), _p(q), C.byref(pe),
                       C.byref(re))
    return pe.value, re.value


def cholesky_solve(A, b):
    A = _f64(A)
    b = _f64(b)
    n = b.shape[0]
    x = np.empty(n)
    rc = lib().or_cholesky_solve(n, A.ctypes.data_as(_f64p), _p(b), _p(x))
    return x if rc == 0 else None


def ik_solve(robot: Robot, params: IkParams, tg: Targets, targets, seeds, n_trace=0,
             per_problem=False, n_threads=0):
    """Multi-start LM.  targets [B][k][12], seeds [B][S][n_dof].

    Returns a dict with q [B][n], err [B][2], iters [B], status [B], threads, and
    (optionally) per_problem [B*S][n+5], trace [B*S][n_trace][n], margin [B*S].
    """
    targets = _f64(targets).reshape(-1, tg.k, 12)
    B = targets.shape[0]
    seeds = _f64(seeds).reshape(B, -1, robot.n_dof)
    S = seeds.shape[1]
    n = robot.n_dof
    q = np.zeros((B, n))
    err = np.zeros((B, 2))
    iters = np.zeros(B, np.int32)
    status = np.zeros(B, np.int32)
    pp = np.zeros((B * S, n + 5)) if per_problem else None
    tr = np.zeros((B * S, n_trace, n)) if n_trace > 0 else None
    mg = np.zeros(B * S) if n_trace > 0 else None
    threads = lib().or_ik_solve(
        C.byref(robot._c), C.byref(params._c), C.byref(tg._c), B, S, _p(targets), _p(seeds),
        _p(q), _p(err), _p(iters), _p(status), None if pp is None else pp.ctypes.data_as(_f64p),
        int(n_trace), None if tr is None else tr.ctypes.data_as(_f64p), _p(mg), int(n_threads))
    out = dict(q=q, err=err, iters=iters, status=status, threads=int(threads))
    if pp is not None:
        out["per_problem"] = pp
    if tr is not None:
        out["trace"] = tr
        out["margin"] = mg
    return out


def lm_run(robot: Robot, params: IkParams, tg: Targets, targets, seed, n_trace, lambda_init=-1.0):
    """One LM run of a single problem (targets [k][12], seed [n_dof]) with its
    configuration and damping after iterations 1..n_trace.

    Returns a dict with q [n], q_trace [n_trace][n], lam_trace [n_trace], cost,
    pos_err, rot_err, iters, status and lam (the final damping)."""
    targets = _f64(targets).reshape(tg.k, 12)
    seed = _f64(seed).reshape(robot.n_dof)
    n = robot.n_dof
    qtr = np.zeros((max(n_trace, 1), n))
    ltr = np.zeros(max(n_trace, 1))
    q = np.zeros(n)
    res = np.zeros(6)
    lib().or_lm_run(C.byref(robot._c), C.byref(params._c), C.byref(tg._c), _p(targets), _p(seed),
                    C.c_double(lambda_init), int(n_trace), _p(qtr), _p(ltr), _p(q), _p(res))
    return dict(q=q, q_trace=qtr[:n_trace], lam_trace=ltr[:n_trace], cost=res[0], pos_err=res[1],
                rot_err=res[2], iters=int(res[3]), status=int(res[4]), lam=res[5])


def ik_beam(robot: Robot, params: IkParams, tg: Targets, targets, seeds, steps1=6, keep=4, steps2=10,
            n_threads=0):
    """IK-Beam (Sec. V-C).  targets [B][k][12], seeds [B][S][n_dof]; steps1 LM
    iterations on all S seeds, the `keep` lowest-cost seeds continue for steps2.

    Returns a dict with q [B][n], err [B][2], iters [B], status [B], kept [B][keep]
    (selected seed indices, in selection order) and threads."""
    targets = _f64(targets).reshape(-1, tg.k, 12)
    B = targets.shape[0]
    seeds = _f64(seeds).reshape(B, -1, robot.n_dof)
    S = seeds.shape[1]
    n = robot.n_dof
    q = np.zeros((B, n))
    err = np.zeros((B, 2))
    iters = np.zeros(B, np.int32)
    status = np.zeros(B, np.int32)
    kept = np.zeros((B, keep), np.int32)
    threads = lib().or_ik_beam(C.byref(robot._c), C.byref(params._c), C.byref(tg._c), B, S, int(steps1),
                               int(keep), int(steps2), _p(targets), _p(seeds), _p(q), _p(err), _p(iters),
                               _p(status), _p(kept), int(n_threads))
    return dict(q=q, err=err, iters=iters, status=status, kept=kept, threads=int(threads))


# ---------------------------------------------------------------- FLOP census
def ik_flop_units(robot: Robot, params: IkParams, tg: Targets, targets, q, lam=1e-2):
    """Algorithmic work of the three LM units at configuration q, counted on
    the oracle's own arithmetic (flopcount.hpp): dict(eval, build, solve) of
    (FLOPs, special-function calls)."""
    targets = _f64(targets).reshape(tg.k, 12)
    q = _f64(q)
    out = np.zeros(6, np.int64)
    flops_lib().orf_ik_units(C.byref(robot._c), C.byref(params._c), C.byref(tg._c), _p(targets), _p(q),
                             C.c_double(lam), out.ctypes.data_as(C.POINTER(C.c_int64)))
    return dict(eval=(int(out[0]), int(out[1])), build=(int(out[2]), int(out[3])), solve=(int(out[4]), int(out[5])))


# ---------------------------------------------------------------- seed network
def mlp_n_params(dims):
    return int(sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1)))


def mlp_forward(dims, params, x):
    """Pre-head outputs [M][dims[-1]] of the SiLU MLP (FP64)."""
    dims_a = _i32(dims)
    params = _f64(params)
    x = _f64(x).reshape(-1, dims[0])
    y = np.empty((x.shape[0], dims[-1]))
    lib().or_mlp_forward(len(dims) - 1, _p(dims_a), _p(params), x.shape[0], _p(x), _p(y))
    return y


def round_bf16(x):
    """x rounded to BF16 (8 significant bits, ties to even), as float64."""
    x = _f64(x)
    y = np.empty_like(x)
    lib().or_round_bf16(C.c_int64(x.size), _p(x), _p(y))
    return y


def mlp_forward_bf16(dims, params, x):
    """Pre-head outputs [M][dims[-1]] at the network's own precision (BF16
    operands into every layer: hidden SiLU outputs rounded to BF16; FP64 sums)
    and the output layer's magnitude scale sum |W||a| + |b| [M][dims[-1]]."""
    dims_a = _i32(dims)
    params = _f64(params)
    x = _f64(x).reshape(-1, dims[0])
    y = np.empty((x.shape[0], dims[-1]))
    sc = np.empty((x.shape[0], dims[-1]))
    lib().or_mlp_forward_bf16(len(dims) - 1, _p(dims_a), _p(params), x.shape[0], _p(x), _p(y), _p(sc))
    return y, sc


def mlp_loss_grad(dims, params, x, q_star, K, lo, hi, mu=0.01):
    """(mean loss, gradient [n_params], proposals [M][K][n]) of the min-over-K loss."""
    dims_a = _i32(dims)
    params = _f64(params)
    x = _f64(x).reshape(-1, dims[0])
    M = x.shape[0]
    q_star = _f64(q_star).reshape(M, -1)
    n = q_star.shape[1]
    grad = np.empty(mlp_n_params(dims))
    q = np.empty((M, K, n))
    loss = C.c_double()
    rc = lib().or_mlp_loss_grad(len(dims) - 1, _p(dims_a), _p(params), M, _p(x), _p(q_star), K, n,
                                _p(_f64(lo)), _p(_f64(hi)), C.c_double(mu), _p(grad), _p(q),
                                C.byref(loss))
    if rc != 0:
        raise ValueError("last layer width must be K * n")
    return loss.value, grad, q


def adamw(p, g, m, v, lr, beta1, beta2, eps, wd, step):
    """One AdamW step in place on FP64 arrays p, m, v."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().or_adamw(C.c_int64(p.size), _p(p), _p(g), _p(m), _p(v), C.c_double(lr), C.c_double(beta1),
                   C.c_double(beta2), C.c_double(eps), C.c_double(wd), C.c_int64(step))


# ---------------------------------------------------------------- trajectory optimisation
class _TrajParams(C.Structure):
    _fields_ = [("w_start", C.c_double), ("w_goal_pos", C.c_double), ("w_goal_rot", C.c_double),
                ("w_vel", C.c_double), ("w_acc", C.c_double), ("w_limit", C.c_double),
                ("w_coll", C.c_double), ("eta", C.c_double), ("lambda0", C.c_double),
                ("lambda_min", C.c_double), ("lambda_max", C.c_double), ("nu", C.c_double),
                ("iters", C.c_int32), ("banded", C.c_int32), ("w_vlimit", C.c_double), ("v_max", C.c_double),
                ("w_swept", C.c_double), ("w_acc5", C.c_double), ("w_jerk", C.c_double)]


class _TrajScene(C.Structure):
    _fields_ = [("S", C.c_int32), ("radii", _f64p), ("n_obs", C.c_int32), ("obs", _f64p),
                ("plane", _f64p)]


class TrajParams:
    def __init__(self, w_start=100.0, w_goal_pos=100.0, w_goal_rot=50.0, w_vel=1.0, w_acc=1.0, w_limit=10.0,
                 w_coll=10.0, eta=0.02, lambda0=1e-2, lambda_min=1e-10, lambda_max=1e10, nu=2.0, iters=50,
                 banded=1, w_vlimit=0.0, v_max=0.1, w_swept=0.0, w_acc5=0.0, w_jerk=0.0):
        self._c = _TrajParams(w_start, w_goal_pos, w_goal_rot, w_vel, w_acc, w_limit, w_coll, eta, lambda0,
                              lambda_min, lambda_max, nu, iters, banded, w_vlimit, v_max, w_swept, w_acc5, w_jerk)

    def __getattr__(self, k):
        return getattr(self.__dict__["_c"], k)


class Scene:
    """Link spheres (radii [n_dof][S]), obstacles [n_obs][4] and a plane [4]."""

    def __init__(self, radii, obstacles, plane):
        self.radii = _f64(radii)
        self.obs = _f64(obstacles).reshape(-1, 4)
        self.plane = _f64(plane)
        self._c = _TrajScene(int(self.radii.shape[1]), _p(self.radii), int(self.obs.shape[0]),
                             _p(self.obs) if self.obs.size else None, _p(self.plane))


def coll_activation(d, eta):
    df = C.c_double()
    f = lib().or_coll_activation(C.c_double(d), C.c_double(eta), C.byref(df))
    return f, df.value


def traj_n_residuals(robot, scene, T):
    return int(lib().or_traj_n_residuals(C.byref(robot._c), C.byref(scene._c), T))


def traj_residual(robot, params, scene, x, q_start, goal, jacobian=True):
    x = _f64(x)
    T = x.shape[0]
    m = traj_n_residuals(robot, scene, T)
    r = np.empty(m)
    J = np.empty((m, x.size)) if jacobian else None
    lib().or_traj_residual(C.byref(robot._c), C.byref(params._c), C.byref(scene._c), T, _p(x),
                           _p(_f64(q_start)), _p(_f64(goal)), _p(r), None if J is None else J.ctypes.data_as(_f64p))
    return (r, J) if jacobian else r


def traj_normal(robot, params, scene, x, q_start, goal):
    x = _f64(x)
    N = x.size
    A = np.empty((N, N))
    g = np.empty(N)
    f = lib().or_traj_normal(C.byref(robot._c), C.byref(params._c), C.byref(scene._c), x.shape[0], _p(x),
                             _p(_f64(q_start)), _p(_f64(goal)), A.ctypes.data_as(_f64p), _p(g))
    return f, A, g


def banded_cholesky(A, T, n, band=2):
    A = _f64(A)
    L = np.empty_like(A)
    rc = lib().or_banded_cholesky_b(T, n, band, A.ctypes.data_as(_f64p), L.ctypes.data_as(_f64p))
    return L if rc == 0 else None


def traj_lm_run(robot, params, scene, x0, q_start, goal):
    """One trajectory's LM run (x0 [T][n]).  Returns dict(x, cost, trace
    [iters][T][n], lam_trace [iters]): x and the damping after every iteration."""
    x = _f64(x0).copy()
    T, n = x.shape
    tr = np.empty((params.iters, T, n))
    lt = np.empty(params.iters)
    f = lib().or_traj_lm_run(C.byref(robot._c), C.byref(params._c), C.byref(scene._c), T, _p(x),
                             _p(_f64(q_start)), _p(_f64(goal)), tr.ctypes.data_as(_f64p), _p(lt))
    return dict(x=x, cost=f, trace=tr, lam_trace=lt)


def traj_flop_units(robot, params, scene, x, q_start, goal, lam=1e-2):
    """Algorithmic work of one trajectory's LM units at x [T][n], counted on
    the oracle's own arithmetic: dict(eval, build, solve) of (FLOPs, special
    calls)."""
    x = _f64(x)
    out = np.zeros(6, np.int64)
    flops_lib().orf_traj_units(C.byref(robot._c), C.byref(params._c), C.byref(scene._c), x.shape[0], _p(x),
                               _p(_f64(q_start)), _p(_f64(goal)), C.c_double(lam),
                               out.ctypes.data_as(C.POINTER(C.c_int64)))
    return dict(eval=(int(out[0]), int(out[1])), build=(int(out[2]), int(out[3])), solve=(int(out[4]), int(out[5])))


def traj_solve(robot, params, scene, x0, q_start, goals, n_trace=False, n_threads=0):
    """Batched LM; x0 [B][T][n].  Returns dict(x, cost, threads[, trace, margin])."""
    x = _f64(x0).copy()
    B, T, n = x.shape
    cost = np.empty(B)
    tr = np.empty((B, params.iters, T, n)) if n_trace else None
    mg = np.empty(B) if n_trace else None
    thr = lib().or_traj_solve(C.byref(robot._c), C.byref(params._c), C.byref(scene._c), B, T, _p(x),
                              _p(_f64(q_start)), _p(_f64(goals)), _p(cost),
                              None if tr is None else tr.ctypes.data_as(_f64p), _p(mg), int(n_threads))
    out = dict(x=x, cost=cost, threads=int(thr))
    if tr is not None:
        out["trace"] = tr
        out["margin"] = mg
    return out
