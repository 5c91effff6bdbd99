"""Python binding of libpk (include/pk.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it checks tensor devices, dtypes and shapes, passes
``data_ptr()`` values and the current CUDA stream, and turns a non-PK_OK
status into :class:`PkError`.  Device memory comes from PyTorch tensors.

The CUDA library must have been built (``__graft_entry__.build()`` or
``python -m paper_2505_03728_gb300.build``); importing a function that needs it
raises immediately if ``libpk.so`` is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# PK_DEBUG_BOUNDS=1 in the environment selects the index-checked build
# (libpk_debug.so, build(debug_bounds=True)); tests only.
LIB_PATH = os.path.join(HERE, "libpk_debug.so" if os.environ.get("PK_DEBUG_BOUNDS") == "1" else "libpk.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pk.h")

PK_OK, PK_ERR_INVALID_ARG, PK_ERR_CUDA, PK_ERR_OOM, PK_ERR_TIMEOUT, PK_ERR_UNSUPPORTED = range(6)
PK_JOINT_FIXED, PK_JOINT_REVOLUTE, PK_JOINT_PRISMATIC = 0, 1, 2
PK_TARGET_POSE, PK_TARGET_POSITION = 0, 1
PK_P_CONVERGED, PK_P_MAX_ITERS, PK_P_NONFINITE, PK_P_CANCELLED = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


class PkError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libpk status {status}: {message}")
        self.status = status


class pk_ik_params(C.Structure):
    _fields_ = [("w_pos", C.c_float), ("w_rot", C.c_float), ("w_limit", C.c_float),
                ("w_rest", C.c_float), ("lambda0", C.c_float), ("lambda_min", C.c_float),
                ("lambda_max", C.c_float), ("nu", C.c_float), ("tol_pos", C.c_float),
                ("tol_rot", C.c_float), ("max_iters", C.c_int32), ("early_exit", C.c_int32),
                ("cancel_siblings", C.c_int32), ("reserved", C.c_int32), ("w_self", C.c_float),
                ("eta_self", C.c_float)]


class pk_ik_beam_params(C.Structure):
    _fields_ = [("n_seeds", C.c_int32), ("steps1", C.c_int32), ("keep", C.c_int32), ("steps2", C.c_int32)]


class pk_ik_problem_set(C.Structure):
    _fields_ = [("robot", C.c_void_p), ("k", C.c_int32), ("target_links", C.POINTER(C.c_int32)),
                ("target_kinds", C.POINTER(C.c_int32)), ("batch", C.c_int32), ("n_seeds", C.c_int32),
                ("d_targets", C.c_void_p), ("d_seeds", C.c_void_p), ("d_q_out", C.c_void_p),
                ("d_err_out", C.c_void_p), ("d_iters_out", C.c_void_p), ("d_status_out", C.c_void_p)]


class pk_trajopt_params(C.Structure):
    _fields_ = [("w_start", C.c_float), ("w_goal_pos", C.c_float), ("w_goal_rot", C.c_float),
                ("w_vel", C.c_float), ("w_acc", C.c_float), ("w_limit", C.c_float), ("w_coll", C.c_float),
                ("eta", C.c_float), ("lambda0", C.c_float), ("lambda_min", C.c_float),
                ("lambda_max", C.c_float), ("nu", C.c_float), ("tol_pos", C.c_float), ("tol_rot", C.c_float),
                ("iters", C.c_int32), ("reserved", C.c_int32), ("w_vlimit", C.c_float), ("v_max", C.c_float),
                ("w_swept", C.c_float), ("w_acc5", C.c_float), ("w_jerk", C.c_float)]


class pk_train_params(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("steps_per_epoch", C.c_int32),
                ("lr", C.c_float), ("weight_decay", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("mu", C.c_float), ("refine_every", C.c_int32),
                ("seed", C.c_uint64), ("refine_n", C.c_int32), ("refine_iters", C.c_int32),
                ("pool_frac", C.c_float), ("first_epoch", C.c_int32), ("last_epoch", C.c_int32)]


_vp = C.c_void_p
_i32 = C.c_int32
_i32p = C.POINTER(C.c_int32)
_f32p = C.POINTER(C.c_float)

_SIGNATURES = {
    "pk_ik_params_default": (None, [C.POINTER(pk_ik_params)]),
    "pk_last_error": (C.c_char_p, []),
    "pk_robot_create": (_i32, [_i32, _i32p, _i32p, _f32p, _f32p, _f32p, _f32p, _f32p, C.POINTER(_vp)]),
    "pk_robot_destroy": (None, [_vp]),
    "pk_robot_n_joints": (_i32, [_vp]),
    "pk_robot_n_dof": (_i32, [_vp]),
    "pk_robot_set_mimic": (_i32, [_vp, _i32, _i32, C.c_float, C.c_float]),
    "pk_robot_set_spheres": (_i32, [_vp, _i32, _i32p, _f32p, _f32p, _i32, _i32p]),
    "pk_fk": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "pk_ik_residual": (_i32, [_vp, C.POINTER(pk_ik_params), _i32, _i32p, _i32p, _i32, _vp, _vp, _vp,
                              _vp, _vp]),
    "pk_ik_workspace_bytes": (C.c_size_t, [_vp, _i32, _i32]),
    "pk_ik_beam_params_default": (None, [C.POINTER(pk_ik_beam_params)]),
    "pk_ik_beam_workspace_bytes": (C.c_size_t, [_vp, _i32, C.POINTER(pk_ik_beam_params)]),
    "pk_ik_beam_solve": (_i32, [_vp, C.POINTER(pk_ik_params), C.POINTER(pk_ik_beam_params), _i32, _i32p, _i32p,
                                _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "pk_ik_solve": (_i32, [_vp, C.POINTER(pk_ik_params), _i32, _i32p, _i32p, _i32, _i32, _vp, _vp,
                           _vp, _vp, _vp, _vp, _vp, C.c_size_t, _vp]),
    "pk_ik_split_workspace_bytes": (C.c_size_t, [_vp, _i32, _i32]),
    "pk_ik_solve_split": (_i32, [_vp, C.POINTER(pk_ik_params), _i32, _i32p, _i32p, _i32, _i32, _vp, _vp,
                                 _vp, _vp, _vp, _vp, _vp, C.c_size_t, _i32, _i32, _vp, _vp]),
    "pk_ik_solve_noalloc": (_i32, [_vp, C.POINTER(pk_ik_params), _i32, _i32p, _i32p, _i32, _i32, _vp,
                                   _vp, _vp, _vp, _vp, _vp, _vp]),
    "pk_ik_workspace_stats": (_i32, [_vp, C.POINTER(C.c_int64)]),
    "pk_ik_split_workspace_stats": (_i32, [_vp, C.POINTER(C.c_int64)]),
    "pk_train_params_default": (None, [_vp]),
    "pk_ik_plan_create": (_i32, [C.POINTER(pk_ik_params), _i32, _vp, C.POINTER(_vp)]),
    "pk_ik_plan_destroy": (None, [_vp]),
    "pk_ik_plan_run": (_i32, [_vp, _vp]),
    "pk_ik_plan_run_eager": (_i32, [_vp, _vp]),
    "pk_ik_plan_autotune": (_i32, [_vp, _i32, _vp, C.POINTER(C.c_float)]),
    "pk_ik_plan_schedule": (_i32, [_vp, _i32p, _i32p, _i32p, _i32p, _i32p]),
    "pk_ik_plan_set_schedule": (_i32, [_vp, _i32, _i32, _i32, _i32]),
    "pk_ik_plan_stats": (_i32, [_vp, C.POINTER(C.c_int64)]),
    "pk_seednet_check": (_i32, [_vp, _vp]),
    "pk_seednet_save": (_i32, [_vp, C.c_char_p]),
    "pk_seednet_load": (_i32, [_vp, C.c_char_p]),
    "pk_trajopt_params_default": (None, [_vp]),
    "pk_trajopt_solve": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _vp, _i32, _vp, _i32, _vp, _f32p, _vp, _vp,
                                _vp, _vp]),
    "pk_trajopt_normal": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _vp, _i32, _vp, _i32, _vp, _f32p, _vp, _vp, _vp,
                                 _vp, _vp]),
    "pk_trajopt_interpolate": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp, _vp]),
    "pk_ik_select_clear": (_i32, [_vp, _i32, _i32, _vp, _i32, _vp, _i32, _vp, _f32p, C.c_float, _vp, _vp, _vp, _vp,
                                  _vp]),
    "pk_seednet_create": (_i32, [_vp, _i32, _i32p, _i32, _i32, _i32, C.c_uint64, C.POINTER(_vp)]),
    "pk_seednet_destroy": (None, [_vp]),
    "pk_seednet_n_params": (C.c_int64, [_vp]),
    "pk_seednet_get_params": (_i32, [_vp, _f32p, C.c_int64]),
    "pk_seednet_set_params": (_i32, [_vp, _f32p, C.c_int64]),
    "pk_seednet_forward": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "pk_seednet_infer": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "pk_seednet_loss_grad": (_i32, [_vp, _i32, _vp, _vp, _f32p, _f32p, _vp]),
    "pk_seednet_train_step": (_i32, [_vp, _vp, _i32, _vp, _vp, C.c_float, _vp]),
    "pk_seednet_train": (_i32, [_vp, _vp, _f32p, _vp]),
    "pk_seednet_refine": (_i32, [_vp, _i32, _i32, C.c_uint64, _i32p, _vp]),
    "pk_seednet_pool": (_i32, [_vp, _vp, _vp, _i32p, _vp]),
    "pk_trace_enable": (_i32, [_i32]),
    "pk_debug_bounds_enabled": (_i32, []),
    "pk_debug_bounds_take": (_i32, [C.POINTER(C.c_uint64)]),
    "pk_debug_bounds_selftest": (_i32, [_i32, _vp]),
    "pk_trace_summary": (_i32, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
}


def lib():
    """The loaded libpk.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                                   "(python -m paper_2505_03728_gb300.build)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGNATURES.items():
                if hasattr(L, name):
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
            _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of every function declared in include/pk.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pk_[a-z0-9_]+)\s*\(", text)))


def _check(status):
    if status != PK_OK:
        raise PkError(status, pk_last_error())


def pk_last_error() -> str:
    return lib().pk_last_error().decode()


def pk_ik_params_default(**overrides) -> pk_ik_params:
    p = pk_ik_params()
    lib().pk_ik_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t, dtype=torch.float32, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


class Robot:
    """Owns a pk_robot handle (pk_robot_create / pk_robot_destroy)."""

    def __init__(self, parent, type, axis, origin, lower, upper, tool=None):
        parent = np.ascontiguousarray(parent, np.int32)
        type = np.ascontiguousarray(type, np.int32)
        axis = np.ascontiguousarray(axis, np.float32).reshape(-1)
        origin = np.ascontiguousarray(origin, np.float32).reshape(-1)
        lower = np.ascontiguousarray(lower, np.float32)
        upper = np.ascontiguousarray(upper, np.float32)
        tool_p = None
        if tool is not None:
            tool = np.ascontiguousarray(tool, np.float32)
            tool_p = tool.ctypes.data_as(_f32p)
        h = C.c_void_p()
        _check(lib().pk_robot_create(len(parent), parent.ctypes.data_as(_i32p),
                                     type.ctypes.data_as(_i32p), axis.ctypes.data_as(_f32p),
                                     origin.ctypes.data_as(_f32p), lower.ctypes.data_as(_f32p),
                                     upper.ctypes.data_as(_f32p), tool_p, C.byref(h)))
        self.handle = h
        self.n_joints = lib().pk_robot_n_joints(h)
        self.n_dof = lib().pk_robot_n_dof(h)

    def set_mimic(self, joint: int, source: int, multiplier: float = 1.0, offset: float = 0.0):
        """Make `joint` follow `source`'s variable: value = multiplier * q_source + offset."""
        _check(lib().pk_robot_set_mimic(self.handle, int(joint), int(source), C.c_float(multiplier),
                                        C.c_float(offset)))
        self.n_dof = lib().pk_robot_n_dof(self.handle)

    def set_spheres(self, joint, centre, radius, pairs):
        """Self-collision model: spheres (frame, centre in it, radius) and the pairs that must stay apart."""
        joint = np.ascontiguousarray(joint, np.int32).reshape(-1)
        centre = np.ascontiguousarray(centre, np.float32).reshape(-1)
        radius = np.ascontiguousarray(radius, np.float32).reshape(-1)
        pairs = np.ascontiguousarray(pairs, np.int32).reshape(-1)
        _check(lib().pk_robot_set_spheres(self.handle, len(joint), joint.ctypes.data_as(_i32p),
                                          centre.ctypes.data_as(_f32p), radius.ctypes.data_as(_f32p),
                                          len(pairs) // 2, pairs.ctypes.data_as(_i32p)))

    @classmethod
    def from_spec(cls, spec):
        r = cls(spec["parent"], spec["type"], spec["axis"], spec["origin"], spec["lower"], spec["upper"])
        mimic = spec.get("mimic")
        if mimic is not None:
            for j, s in enumerate(np.asarray(mimic)):
                if s >= 0:
                    r.set_mimic(j, int(s), float(spec["mimic_mult"][j]), float(spec["mimic_off"][j]))
        sp = spec.get("spheres")
        if sp is not None:
            r.set_spheres(sp["joint"], sp["centre"], sp["radius"], sp["pairs"])
        return r

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.pk_robot_destroy(h)
            self.handle = None


def _links(links, kinds):
    links = np.ascontiguousarray(links, np.int32).reshape(-1)
    kinds_a = None if kinds is None else np.ascontiguousarray(kinds, np.int32).reshape(-1)
    return links, kinds_a, (None if kinds_a is None else kinds_a.ctypes.data_as(_i32p))


def pk_fk(robot: Robot, q: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """All joint frames [B][n_joints][12] for configurations q [B][n_dof]."""
    B = q.shape[0]
    if q.shape != (B, robot.n_dof):
        raise ValueError("q must be [batch][n_dof]")
    if out is None:
        out = torch.empty(B, robot.n_joints, 12, device=q.device, dtype=torch.float32)
    _check(lib().pk_fk(robot.handle, B, _dev(q, name="q"), _dev(out, name="out"), _stream(stream)))
    return out


def pk_ik_residual(robot: Robot, params: pk_ik_params, links, kinds, targets: torch.Tensor,
                   q: torch.Tensor, jacobian=True, stream=None):
    """Weighted residuals [B][m] and Jacobian [B][m][n_dof] at q [B][n_dof]."""
    links, kinds_a, kinds_p = _links(links, kinds)
    B = q.shape[0]
    rows = 3 if (kinds_a is not None and kinds_a[0] == PK_TARGET_POSITION) else 6
    m = rows * len(links) + 2 * robot.n_dof
    r = torch.empty(B, m, device=q.device, dtype=torch.float32)
    J = torch.empty(B, m, robot.n_dof, device=q.device, dtype=torch.float32) if jacobian else None
    _check(lib().pk_ik_residual(robot.handle, C.byref(params), len(links), links.ctypes.data_as(_i32p),
                                kinds_p, B, _dev(targets, name="targets"), _dev(q, name="q"),
                                _dev(r, name="r"), None if J is None else _dev(J, name="J"),
                                _stream(stream)))
    return (r, J) if jacobian else r


def pk_ik_workspace_bytes(robot: Robot, batch: int, n_seeds: int) -> int:
    return int(lib().pk_ik_workspace_bytes(robot.handle, batch, n_seeds))


def pk_ik_solve(robot: Robot, params: pk_ik_params, links, kinds, targets: torch.Tensor,
                seeds: torch.Tensor, workspace: torch.Tensor | None = None, out=None, stream=None):
    """Multi-start LM IK.  targets [B][k][12], seeds [B][S][n_dof].

    Returns (q [B][n_dof], err [B][2], iters [B], status [B]) as CUDA tensors.
    """
    links, kinds_a, kinds_p = _links(links, kinds)
    B, S = seeds.shape[0], seeds.shape[1]
    if seeds.shape != (B, S, robot.n_dof):
        raise ValueError("seeds must be [batch][n_seeds][n_dof]")
    if targets.shape != (B, len(links), 12):
        raise ValueError("targets must be [batch][k][12]")
    dev = seeds.device
    if out is None:
        out = (torch.empty(B, robot.n_dof, device=dev), torch.empty(B, 2, device=dev),
               torch.empty(B, device=dev, dtype=torch.int32), torch.empty(B, device=dev, dtype=torch.int32))
    q, err, iters, status = out
    ws_p, ws_n = None, 0
    if workspace is not None:
        ws_p, ws_n = _dev(workspace, torch.uint8, "workspace"), workspace.numel()
    _check(lib().pk_ik_solve(robot.handle, C.byref(params), len(links), links.ctypes.data_as(_i32p),
                             kinds_p, B, S, _dev(targets, name="targets"), _dev(seeds, name="seeds"),
                             _dev(q, name="q"), _dev(err, name="err"),
                             _dev(iters, torch.int32, "iters"), _dev(status, torch.int32, "status"),
                             ws_p, ws_n, _stream(stream)))
    return q, err, iters, status


def pk_ik_split_workspace_bytes(robot: Robot, batch: int, n_seeds: int) -> int:
    return int(lib().pk_ik_split_workspace_bytes(robot.handle, batch, n_seeds))


def pk_ik_solve_split(robot: Robot, params: pk_ik_params, links, kinds, targets: torch.Tensor,
                      seeds: torch.Tensor, workspace: torch.Tensor, split_iters: int, tail_ctas: int = 0,
                      out=None, stream=None, tail_stream=None):
    """pk_ik_solve in two launches: every problem up to ``split_iters``
    iterations on ``stream``, the problems still running then resumed on
    ``tail_stream`` (``tail_ctas`` blocks, 0: full grid), where the outputs
    are complete.  ``workspace``: pk_ik_split_workspace_bytes() bytes."""
    links, kinds_a, kinds_p = _links(links, kinds)
    B, S = seeds.shape[0], seeds.shape[1]
    if seeds.shape != (B, S, robot.n_dof):
        raise ValueError("seeds must be [batch][n_seeds][n_dof]")
    if targets.shape != (B, len(links), 12):
        raise ValueError("targets must be [batch][k][12]")
    dev = seeds.device
    if out is None:
        out = (torch.empty(B, robot.n_dof, device=dev), torch.empty(B, 2, device=dev),
               torch.empty(B, device=dev, dtype=torch.int32), torch.empty(B, device=dev, dtype=torch.int32))
    q, err, iters, status = out
    st = _stream(stream)
    tst = st if tail_stream is None else _stream(tail_stream)
    _check(lib().pk_ik_solve_split(robot.handle, C.byref(params), len(links), links.ctypes.data_as(_i32p),
                                   kinds_p, B, S, _dev(targets, name="targets"), _dev(seeds, name="seeds"),
                                   _dev(q, name="q"), _dev(err, name="err"),
                                   _dev(iters, torch.int32, "iters"), _dev(status, torch.int32, "status"),
                                   _dev(workspace, torch.uint8, "workspace"), workspace.numel(), split_iters,
                                   tail_ctas, st, tst))
    return q, err, iters, status


def pk_ik_beam_params_default(**overrides) -> pk_ik_beam_params:
    b = pk_ik_beam_params()
    lib().pk_ik_beam_params_default(C.byref(b))
    for k, v in overrides.items():
        setattr(b, k, v)
    return b


def pk_ik_beam_workspace_bytes(robot: Robot, batch: int, beam: pk_ik_beam_params) -> int:
    return int(lib().pk_ik_beam_workspace_bytes(robot.handle, batch, C.byref(beam)))


def pk_ik_beam_solve(robot: Robot, params: pk_ik_params, beam: pk_ik_beam_params, links, kinds,
                     targets: torch.Tensor, seeds: torch.Tensor, workspace: torch.Tensor | None = None,
                     out=None, kept: torch.Tensor | None = None, stream=None):
    """IK-Beam.  targets [B][1][12], seeds [B][beam.n_seeds][n_dof].

    Returns (q [B][n_dof], err [B][2], iters [B], status [B]) as CUDA tensors;
    ``kept`` ([B][beam.keep] int32), when given, receives the kept seed indices.
    """
    links, kinds_a, kinds_p = _links(links, kinds)
    B = seeds.shape[0]
    if seeds.shape != (B, beam.n_seeds, robot.n_dof):
        raise ValueError("seeds must be [batch][beam.n_seeds][n_dof]")
    if targets.shape != (B, len(links), 12):
        raise ValueError("targets must be [batch][k][12]")
    dev = seeds.device
    if out is None:
        out = (torch.empty(B, robot.n_dof, device=dev), torch.empty(B, 2, device=dev),
               torch.empty(B, device=dev, dtype=torch.int32), torch.empty(B, device=dev, dtype=torch.int32))
    q, err, iters, status = out
    ws_p, ws_n = None, 0
    if workspace is not None:
        ws_p, ws_n = _dev(workspace, torch.uint8, "workspace"), workspace.numel()
    kept_p = None if kept is None else _dev(kept, torch.int32, "kept")
    _check(lib().pk_ik_beam_solve(robot.handle, C.byref(params), C.byref(beam), len(links),
                                  links.ctypes.data_as(_i32p), kinds_p, B, _dev(targets, name="targets"),
                                  _dev(seeds, name="seeds"), _dev(q, name="q"), _dev(err, name="err"),
                                  _dev(iters, torch.int32, "iters"), _dev(status, torch.int32, "status"),
                                  kept_p, ws_p, ws_n, _stream(stream)))
    return q, err, iters, status


def pk_ik_workspace_stats(workspace: torch.Tensor) -> dict:
    """Work counters of the last solve that used ``workspace`` (synchronises)."""
    out = (C.c_int64 * 4)()
    _check(lib().pk_ik_workspace_stats(_dev(workspace, torch.uint8, "workspace"), out))
    return dict(evals=out[0], builds=out[1], solves=out[2], problems=out[3])


def pk_ik_split_workspace_stats(workspace: torch.Tensor) -> tuple:
    """Work counters of the two launches of the last pk_ik_solve_split that
    used ``workspace`` (synchronises): (first launch, second launch)."""
    out = (C.c_int64 * 8)()
    _check(lib().pk_ik_split_workspace_stats(_dev(workspace, torch.uint8, "workspace"), out))
    return tuple(dict(evals=out[i], builds=out[i + 1], solves=out[i + 2], problems=out[i + 3]) for i in (0, 4))


def pk_debug_bounds_enabled() -> bool:
    return bool(lib().pk_debug_bounds_enabled())


def pk_debug_bounds_take() -> int:
    """First failed index check since the last call (0: none), cleared on read."""
    code = C.c_uint64(0)
    _check(lib().pk_debug_bounds_take(C.byref(code)))
    return int(code.value)


def pk_debug_bounds_decode(code: int) -> tuple[int, int, int]:
    """(site, bound, index) of a code from pk_debug_bounds_take; index -1 if negative."""
    site, bound, index = (code >> 48) & 0x7FFF, (code >> 24) & 0xFFFFFF, code & 0xFFFFFF
    return site, bound, (-1 if index == 0xFFFFFF else index)


def pk_debug_bounds_selftest(n: int, stream=None):
    _check(lib().pk_debug_bounds_selftest(int(n), _stream(stream)))


def pk_trace_enable(enable: bool = True):
    _check(lib().pk_trace_enable(1 if enable else 0))


def pk_trace_summary(kernel: str):
    """(total ms, launches) of the traced launches of one kernel family."""
    ms, n = C.c_double(), C.c_int64()
    _check(lib().pk_trace_summary(kernel.encode(), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def pk_ik_solve_noalloc(robot: Robot, params: pk_ik_params, links, kinds, targets: torch.Tensor,
                        seeds: torch.Tensor, out=None, stream=None):
    """pk_ik_solve with the library's static device scratch (no allocation in
    the call).  Same outputs as :func:`pk_ik_solve`."""
    links, kinds_a, kinds_p = _links(links, kinds)
    B, S = seeds.shape[0], seeds.shape[1]
    if seeds.shape != (B, S, robot.n_dof):
        raise ValueError("seeds must be [batch][n_seeds][n_dof]")
    if targets.shape != (B, len(links), 12):
        raise ValueError("targets must be [batch][k][12]")
    dev = seeds.device
    if out is None:
        out = (torch.empty(B, robot.n_dof, device=dev), torch.empty(B, 2, device=dev),
               torch.empty(B, device=dev, dtype=torch.int32), torch.empty(B, device=dev, dtype=torch.int32))
    q, err, iters, status = out
    _check(lib().pk_ik_solve_noalloc(robot.handle, C.byref(params), len(links),
                                     links.ctypes.data_as(_i32p), kinds_p, B, S,
                                     _dev(targets, name="targets"), _dev(seeds, name="seeds"),
                                     _dev(q, name="q"), _dev(err, name="err"),
                                     _dev(iters, torch.int32, "iters"),
                                     _dev(status, torch.int32, "status"), _stream(stream)))
    return q, err, iters, status


def pk_train_params_default(**overrides) -> pk_train_params:
    p = pk_train_params()
    lib().pk_train_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class SeedNet:
    """Owns a pk_seednet handle (pk_seednet_create / pk_seednet_destroy)."""

    def __init__(self, robot: Robot, links, K=8, width=512, depth=4, seed=0):
        links = np.ascontiguousarray(links, np.int32).reshape(-1)
        h = C.c_void_p()
        _check(lib().pk_seednet_create(robot.handle, len(links), links.ctypes.data_as(_i32p), K, width,
                                       depth, seed, C.byref(h)))
        self.handle = h
        self.robot = robot
        self.k, self.K, self.n = len(links), K, robot.n_dof
        self.width, self.depth = width, depth

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.pk_seednet_destroy(h)
            self.handle = None

    @property
    def dims(self):
        return [9 * self.k] + [self.width] * self.depth + [self.K * self.n]


def pk_seednet_n_params(net: SeedNet) -> int:
    return int(lib().pk_seednet_n_params(net.handle))


def pk_seednet_get_params(net: SeedNet) -> np.ndarray:
    out = np.empty(pk_seednet_n_params(net), np.float32)
    _check(lib().pk_seednet_get_params(net.handle, out.ctypes.data_as(_f32p), out.size))
    return out


def pk_seednet_set_params(net: SeedNet, params) -> None:
    params = np.ascontiguousarray(params, np.float32)
    _check(lib().pk_seednet_set_params(net.handle, params.ctypes.data_as(_f32p), params.size))


def pk_seednet_forward(net: SeedNet, targets: torch.Tensor, stream=None) -> torch.Tensor:
    B = targets.shape[0]
    y = torch.empty(B, net.K * net.n, device=targets.device)
    _check(lib().pk_seednet_forward(net.handle, B, _dev(targets, name="targets"), _dev(y, name="y"),
                                    _stream(stream)))
    return y


def pk_seednet_infer(net: SeedNet, targets: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    B = targets.shape[0]
    if out is None:
        out = torch.empty(B, net.K, net.n, device=targets.device)
    _check(lib().pk_seednet_infer(net.handle, B, _dev(targets, name="targets"), _dev(out, name="seeds"),
                                  _stream(stream)))
    return out


def pk_seednet_check(net: SeedNet, stream=None):
    """Synchronise and raise PkError (PK_ERR_TIMEOUT) for a device-side pipeline failure of earlier calls."""
    _check(lib().pk_seednet_check(net.handle, _stream(stream)))


def pk_seednet_save(net: SeedNet, path: str):
    """Write the network's parameters to ``path`` (shape header + FP32 parameters)."""
    _check(lib().pk_seednet_save(net.handle, os.fsencode(path)))


def pk_seednet_load(net: SeedNet, path: str):
    """Read parameters written by pk_seednet_save into a network of the same shape."""
    _check(lib().pk_seednet_load(net.handle, os.fsencode(path)))


def pk_seednet_loss_grad(net: SeedNet, targets: torch.Tensor, qstar: torch.Tensor, stream=None):
    B = targets.shape[0]
    loss = C.c_float()
    grad = np.empty(pk_seednet_n_params(net), np.float32)
    _check(lib().pk_seednet_loss_grad(net.handle, B, _dev(targets, name="targets"), _dev(qstar, name="qstar"),
                                      C.byref(loss), grad.ctypes.data_as(_f32p), _stream(stream)))
    return loss.value, grad


def pk_seednet_train_step(net: SeedNet, params: pk_train_params, targets, qstar, lr: float, stream=None):
    _check(lib().pk_seednet_train_step(net.handle, C.byref(params), targets.shape[0],
                                       _dev(targets, name="targets"), _dev(qstar, name="qstar"),
                                       C.c_float(lr), _stream(stream)))


def pk_seednet_train(net: SeedNet, params: pk_train_params, stream=None) -> np.ndarray:
    """Mean loss of every epoch the call runs (first_epoch .. last_epoch - 1 of the schedule)."""
    last = params.last_epoch if params.last_epoch > 0 else params.epochs
    n = max(0, last - params.first_epoch)
    losses = np.zeros(max(1, n), np.float32)
    _check(lib().pk_seednet_train(net.handle, C.byref(params), losses.ctypes.data_as(_f32p),
                                  _stream(stream)))
    return losses[:n]


def pk_seednet_refine(net: SeedNet, n: int, max_iters: int = 20, seed: int = 500, stream=None) -> int:
    """One LM refinement round of the label pool; returns the converged count."""
    c = C.c_int32()
    _check(lib().pk_seednet_refine(net.handle, n, max_iters, seed, C.byref(c), _stream(stream)))
    return c.value


def pk_seednet_pool(net: SeedNet, stream=None):
    """(targets [n][k][12], labels [n][n_dof]) of the label pool (CUDA tensors)."""
    cnt = C.c_int32()
    _check(lib().pk_seednet_pool(net.handle, None, None, C.byref(cnt), _stream(stream)))
    T = torch.empty(cnt.value, net.k, 12, device="cuda")
    q = torch.empty(cnt.value, net.n, device="cuda")
    if cnt.value:
        _check(lib().pk_seednet_pool(net.handle, _dev(T, name="targets"), _dev(q, name="labels"), C.byref(cnt),
                                     _stream(stream)))
    return T, q


PK_T_OK, PK_T_GOAL_MISSED, PK_T_COLLISION = 0, 1, 2


def pk_trajopt_params_default(**overrides) -> pk_trajopt_params:
    p = pk_trajopt_params()
    lib().pk_trajopt_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _scene_args(radii, obstacles, plane):
    S = radii.shape[1]
    n_obs = obstacles.shape[0]
    pl = np.ascontiguousarray(plane, np.float32)
    return S, n_obs, pl


def pk_trajopt_solve(robot: Robot, params: pk_trajopt_params, q_start, goals, q_init, radii, obstacles, plane,
                     stream=None):
    """Trajectories [B][T][n], costs [B], status bits [B]."""
    B, T, n = q_init.shape
    S, n_obs, pl = _scene_args(radii, obstacles, plane)
    q_out = torch.empty_like(q_init)
    cost = torch.empty(B, device=q_init.device)
    status = torch.empty(B, dtype=torch.int32, device=q_init.device)
    _check(lib().pk_trajopt_solve(robot.handle, C.byref(params), B, T, _dev(q_start, name="q_start"),
                                  _dev(goals, name="goals"), _dev(q_init, name="q_init"), S,
                                  _dev(radii, name="radii"), n_obs,
                                  _dev(obstacles, name="obstacles") if n_obs else None,
                                  pl.ctypes.data_as(_f32p), _dev(q_out, name="q_out"), _dev(cost, name="cost"),
                                  _dev(status, torch.int32, "status"), _stream(stream)))
    return q_out, cost, status


def pk_ik_select_clear(robot: Robot, workspace: torch.Tensor, n_seeds: int, radii, obstacles, plane, margin: float,
                       out, stream=None):
    """Re-choose the answers of the preceding pk_ik_solve (same workspace) preferring converged seeds whose
    link spheres clear the scene by `margin`.  out = (q, err, iters, status) as pk_ik_solve's."""
    q, err, iters, status = out
    B = q.shape[0]
    S, n_obs, pl = _scene_args(radii, obstacles, plane)
    _check(lib().pk_ik_select_clear(robot.handle, B, int(n_seeds), _dev(workspace, torch.uint8, "workspace"), S,
                                    _dev(radii, name="radii"), n_obs,
                                    _dev(obstacles, name="obstacles") if n_obs else None, pl.ctypes.data_as(_f32p),
                                    float(margin), _dev(q, name="q"), _dev(err, name="err"),
                                    _dev(iters, torch.int32, "iters"), _dev(status, torch.int32, "status"),
                                    _stream(stream)))
    return out


def pk_trajopt_interpolate(q_start: torch.Tensor, q_goal: torch.Tensor, T: int, out=None, stream=None):
    """Initial trajectories [B][T][n]: q_start and q_goal [B][n] joined linearly in joint space."""
    B, n = q_start.shape
    if q_goal.shape != (B, n):
        raise ValueError("q_goal must match q_start [batch][n]")
    if out is None:
        out = torch.empty(B, T, n, device=q_start.device)
    _check(lib().pk_trajopt_interpolate(B, int(T), n, _dev(q_start, name="q_start"), _dev(q_goal, name="q_goal"),
                                        _dev(out, name="out"), _stream(stream)))
    return out


def pk_trajopt_normal(robot: Robot, params: pk_trajopt_params, q_start, goals, q, radii, obstacles, plane,
                      stream=None, with_offdiag=False):
    """Diagonal blocks [B][T][n][n], J^T r [B][T][n] and costs [B] at trajectories q
    (and the (t, t-1) blocks [B][T][n][n] last when with_offdiag)."""
    B, T, n = q.shape
    S, n_obs, pl = _scene_args(radii, obstacles, plane)
    D = torch.empty(B, T, n, n, device=q.device)
    E = torch.empty(B, T, n, n, device=q.device) if with_offdiag else None
    g = torch.empty(B, T, n, device=q.device)
    cost = torch.empty(B, device=q.device)
    _check(lib().pk_trajopt_normal(robot.handle, C.byref(params), B, T, _dev(q_start, name="q_start"),
                                   _dev(goals, name="goals"), _dev(q, name="q"), S, _dev(radii, name="radii"),
                                   n_obs, _dev(obstacles, name="obstacles") if n_obs else None,
                                   pl.ctypes.data_as(_f32p), _dev(D, name="D"),
                                   _dev(E, name="E") if E is not None else None, _dev(g, name="g"),
                                   _dev(cost, name="cost"), _stream(stream)))
    return (D, g, cost, E) if with_offdiag else (D, g, cost)


class IkPlan:
    """A pk_ik_plan over several (robot, links, kinds, targets, seeds) sets; keeps
    the tensors it was built on alive and owns the per-set outputs."""

    def __init__(self, params: pk_ik_params, sets):
        self.keep, self.outs = [], []
        arr = (pk_ik_problem_set * len(sets))()
        for i, (robot, links, kinds, targets, seeds) in enumerate(sets):
            links_a, kinds_a, kinds_p = _links(links, kinds)
            B, S = seeds.shape[0], seeds.shape[1]
            dev = seeds.device
            out = (torch.empty(B, robot.n_dof, device=dev), torch.empty(B, 2, device=dev),
                   torch.empty(B, device=dev, dtype=torch.int32), torch.empty(B, device=dev, dtype=torch.int32))
            self.outs.append(out)
            self.keep += [robot, links_a, kinds_a, targets, seeds]
            arr[i] = pk_ik_problem_set(robot.handle.value, len(links_a), links_a.ctypes.data_as(_i32p), kinds_p,
                                       B, S, targets.data_ptr(), seeds.data_ptr(), out[0].data_ptr(),
                                       out[1].data_ptr(), out[2].data_ptr(), out[3].data_ptr())
        self.params = params
        h = C.c_void_p()
        _check(lib().pk_ik_plan_create(C.byref(params), len(sets), C.cast(arr, C.c_void_p), C.byref(h)))
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.pk_ik_plan_destroy(h)
            self.handle = None

    def run(self, stream=None, graph=True):
        fn = lib().pk_ik_plan_run if graph else lib().pk_ik_plan_run_eager
        _check(fn(self.handle, _stream(stream)))
        return self.outs

    def autotune(self, reps=3, stream=None) -> float:
        ms = C.c_float()
        _check(lib().pk_ik_plan_autotune(self.handle, reps, _stream(stream), C.byref(ms)))
        return ms.value

    def schedule(self) -> dict:
        v = [C.c_int32() for _ in range(5)]
        _check(lib().pk_ik_plan_schedule(self.handle, *[C.byref(x) for x in v]))
        return dict(block=v[0].value, grid=v[1].value, chains_as_trees=v[2].value, given_order=v[3].value,
                    variant=v[4].value)

    def set_schedule(self, block=128, chains_as_trees=0, given_order=0, variant=0):
        _check(lib().pk_ik_plan_set_schedule(self.handle, block, chains_as_trees, given_order, variant))

    def stats(self) -> dict:
        out = (C.c_int64 * 4)()
        _check(lib().pk_ik_plan_stats(self.handle, out))
        return dict(evals=out[0], builds=out[1], solves=out[2], problems=out[3])
