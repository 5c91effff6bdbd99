"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module draws random numbers and lays them out; it holds none of the
optimiser's arithmetic (no kinematics, no residuals, no solves).  Target poses
are *not* produced here: callers turn the drawn target configurations into
poses with their own forward kinematics (the CUDA path with ``pk_fk``, the
tests with the CPU oracle).

Generator: NumPy's PCG64 (``numpy.random.default_rng(seed)``).

Robots (Sec. III-B variables; workload shapes of the throughput IK, uneven
batch, learned-seed and trajectory workloads):
  * serial chains: joint axes are normalised Gaussian 3-vectors, each origin is
    a pure translation whose direction is uniform on the sphere and whose
    length is uniform in [0.05, 0.4] m, limits +-2.8 rad, and a fixed tool
    frame appended after the last joint (drawn like a link origin);
  * a 24-DoF hand-like tree (3-joint wrist, fingers of 5, 4, 4, 4, 4 joints,
    one fixed fingertip frame per finger);
  * a 30-joint humanoid-like tree (3-joint torso, two 7-joint arms, two 6-joint
    legs, a 1-joint head, fixed end frames on hands, feet and head).
"""
from __future__ import annotations

import numpy as np

JOINT_FIXED, JOINT_REVOLUTE, JOINT_PRISMATIC = 0, 1, 2
TARGET_POSE, TARGET_POSITION = 0, 1

EYE12 = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], dtype=np.float64)


def _unit(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _translation_origin(rng, lo=0.05, hi=0.4):
    o = EYE12.copy()
    d = _unit(rng, 1)[0] * rng.uniform(lo, hi)
    o[3], o[7], o[11] = d
    return o


class RobotSpec(dict):
    """parent, type, axis [n][3], origin [n][12], lower, upper, plus a name."""

    @property
    def n_joints(self):
        return len(self["parent"])

    def _own_var(self):
        own = np.asarray(self["type"]) != JOINT_FIXED
        if self.get("mimic") is not None:
            own &= np.asarray(self["mimic"]) < 0
        return own

    @property
    def n_dof(self):
        return int(np.sum(self._own_var()))

    @property
    def dof_lower(self):
        return np.asarray(self["lower"])[self._own_var()]

    @property
    def dof_upper(self):
        return np.asarray(self["upper"])[self._own_var()]


def _finish(name, parent, types, axis, origin, lower, upper):
    return RobotSpec(name=name, parent=np.asarray(parent, np.int32), type=np.asarray(types, np.int32),
                     axis=np.asarray(axis, np.float64).reshape(-1, 3),
                     origin=np.asarray(origin, np.float64).reshape(-1, 12),
                     lower=np.asarray(lower, np.float64), upper=np.asarray(upper, np.float64))


def chain_robot(seed: int = 100, n_dof: int = 7, limit: float = 2.8, tool: bool = True,
                prismatic: tuple = ()) -> RobotSpec:
    """Serial chain of ``n_dof`` joints (revolute unless listed in ``prismatic``)."""
    rng = np.random.default_rng(seed)
    n = n_dof + (1 if tool else 0)
    parent = np.arange(n) - 1
    types, axis, origin, lower, upper = [], [], [], [], []
    ax = _unit(rng, n_dof)
    for j in range(n_dof):
        pri = j in prismatic
        types.append(JOINT_PRISMATIC if pri else JOINT_REVOLUTE)
        axis.append(ax[j])
        origin.append(_translation_origin(rng))
        lim = 0.5 if pri else limit
        lower.append(-lim)
        upper.append(lim)
    if tool:
        types.append(JOINT_FIXED)
        axis.append([0.0, 0.0, 1.0])
        origin.append(_translation_origin(rng))
        lower.append(0.0)
        upper.append(0.0)
    return _finish(f"chain{n_dof}", parent, types, axis, origin, lower, upper)


def _add_branch(rng, parent_of_first, n_joints, parent, types, axis, origin, lower, upper,
                limit, tip=True):
    prev = parent_of_first
    ax = _unit(rng, n_joints)
    for j in range(n_joints):
        parent.append(prev)
        types.append(JOINT_REVOLUTE)
        axis.append(ax[j])
        origin.append(_translation_origin(rng, 0.02, 0.12) if limit < 2 else _translation_origin(rng))
        lower.append(-limit)
        upper.append(limit)
        prev = len(parent) - 1
    if tip:
        parent.append(prev)
        types.append(JOINT_FIXED)
        axis.append([0.0, 0.0, 1.0])
        origin.append(_translation_origin(rng, 0.02, 0.05) if limit < 2 else _translation_origin(rng))
        lower.append(0.0)
        upper.append(0.0)
        return len(parent) - 1
    return prev


def mobile_base_robot(arm: RobotSpec, extent: float = 10.0) -> RobotSpec:
    """The arm on an SE(2) mobile base: prismatic x, prismatic y and a revolute
    z joint (all at the world origin) ahead of the arm's joints, so that every
    frame is T_world<-base(x, y, theta) T_base<-i.  Base limits +-extent m and
    +-2 pi rad keep the limit hinge inactive in practice."""
    n0 = len(arm["parent"])
    parent = [-1, 0, 1] + [p + 3 if p >= 0 else 2 for p in arm["parent"]]
    types = [JOINT_PRISMATIC, JOINT_PRISMATIC, JOINT_REVOLUTE] + list(arm["type"])
    axis = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]] + [list(a) for a in arm["axis"]]
    eye = [1.0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 1.0, 0]
    origin = [eye, eye, eye] + [list(o) for o in arm["origin"]]
    lower = [-extent, -extent, -2 * np.pi] + list(arm["lower"])
    upper = [extent, extent, 2 * np.pi] + list(arm["upper"])
    assert len(parent) == n0 + 3
    return _finish("mobile_" + arm["name"], parent, types, axis, origin, lower, upper)


def hand_robot(seed: int = 102) -> tuple[RobotSpec, np.ndarray]:
    """24-DoF hand-like tree; returns (robot, fingertip frame indices [5])."""
    rng = np.random.default_rng(seed)
    parent, types, axis, origin, lower, upper = [], [], [], [], [], []
    wrist = _add_branch(rng, -1, 3, parent, types, axis, origin, lower, upper, 1.5, tip=False)
    tips = []
    for nf in (5, 4, 4, 4, 4):
        tips.append(_add_branch(rng, wrist, nf, parent, types, axis, origin, lower, upper, 1.5))
    return _finish("hand24", parent, types, axis, origin, lower, upper), np.asarray(tips, np.int32)


def hand_mimic_robot(seed: int = 102, mult: float = 0.8, off: float = 0.05) -> tuple[RobotSpec, np.ndarray]:
    """The 24-joint hand with the distal joint of every finger coupled to the
    joint before it (value = mult * q_prev + off), as hands' mimic joints are:
    19 variables.  Returns (robot, fingertip frame indices [5])."""
    spec, tips = hand_robot(seed)
    n = len(spec["parent"])
    mimic = -np.ones(n, np.int32)
    for tip in tips:
        distal = int(spec["parent"][tip])
        mimic[distal] = int(spec["parent"][distal])
    spec = RobotSpec(spec)
    spec["name"] = "hand24_mimic"
    spec["mimic"] = mimic
    spec["mimic_mult"] = np.where(mimic >= 0, mult, 1.0)
    spec["mimic_off"] = np.where(mimic >= 0, off, 0.0)
    return spec, tips


def hand_collision_spheres(spec: RobotSpec, tips, radius: float = 0.012) -> dict:
    """Self-collision model of a hand: one sphere per finger link, on the
    link's joint frame at the midpoint towards the next joint, and the pairs of
    same-depth links of neighbouring fingers.  Returns dict(joint, centre,
    radius, pairs)."""
    parent = np.asarray(spec["parent"])
    origin = np.asarray(spec["origin"]).reshape(-1, 12)
    types = np.asarray(spec["type"])
    fingers = []
    for tip in tips:
        chain = []
        j = int(tip)
        while parent[j] >= 0 and not _branch_point(parent, int(parent[j])):
            chain.append(j)
            j = int(parent[j])
        chain.append(j)
        fingers.append(chain[::-1])  # proximal first, ending at the tip frame
    joint, centre, rad, index = [], [], [], []
    for chain in fingers:
        ids = []
        for a, b in zip(chain[:-1], chain[1:]):
            if types[a] == JOINT_FIXED:
                continue
            ids.append(len(joint))
            joint.append(a)
            centre.append(0.5 * origin[b, [3, 7, 11]])
            rad.append(radius)
        index.append(ids)
    pairs = []
    for f in range(len(index) - 1):
        for l in range(min(len(index[f]), len(index[f + 1]))):
            pairs.append((index[f][l], index[f + 1][l]))
    return dict(joint=np.asarray(joint, np.int32), centre=np.asarray(centre), radius=np.asarray(rad),
                pairs=np.asarray(pairs, np.int32))


def _branch_point(parent, j):
    return int(np.sum(parent == j)) > 1


def humanoid_robot(seed: int = 103) -> tuple[RobotSpec, np.ndarray]:
    """30-joint humanoid-like tree; returns (robot, end frames [6]:
    left hand, right hand, left foot, right foot, head, torso)."""
    rng = np.random.default_rng(seed)
    parent, types, axis, origin, lower, upper = [], [], [], [], [], []
    torso = _add_branch(rng, -1, 3, parent, types, axis, origin, lower, upper, 1.0, tip=False)
    ends = []
    for n in (7, 7):
        ends.append(_add_branch(rng, torso, n, parent, types, axis, origin, lower, upper, 2.5))
    for n in (6, 6):
        ends.append(_add_branch(rng, -1, n, parent, types, axis, origin, lower, upper, 2.0))
    ends.append(_add_branch(rng, torso, 1, parent, types, axis, origin, lower, upper, 1.0))
    ends.append(torso)
    return _finish("humanoid30", parent, types, axis, origin, lower, upper), np.asarray(ends, np.int32)


def uniform_q(seed: int, shape, lower, upper) -> np.ndarray:
    """Joint configurations uniform in [lower, upper]: shape + (n_dof,)."""
    rng = np.random.default_rng(seed)
    lower = np.asarray(lower, np.float64)
    upper = np.asarray(upper, np.float64)
    if isinstance(shape, int):
        shape = (shape,)
    u = rng.random(tuple(shape) + (lower.shape[0],))
    return lower + (upper - lower) * u


def batch_sizes(seed: int, count: int, lo: int = 1, hi: int = 4096) -> np.ndarray:
    """Per-robot batch sizes drawn uniformly from {lo..hi}."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=count)


def sphere_obstacles(seed: int, count: int, reach: float, r_lo=0.05, r_hi=0.2) -> np.ndarray:
    """Obstacle spheres [count][4] (x, y, z, radius), centres uniform in a ball of
    radius ``reach`` above the ground plane z = -0.15."""
    rng = np.random.default_rng(seed)
    out = np.zeros((count, 4))
    i = 0
    while i < count:
        c = rng.uniform(-reach, reach, 3)
        if np.linalg.norm(c) > reach or c[2] < 0.0:
            continue
        out[i, :3] = c
        out[i, 3] = rng.uniform(r_lo, r_hi)
        i += 1
    return out


def link_spheres(seed: int, n_dof: int, per_link: int = 4, r_lo=0.03, r_hi=0.08) -> np.ndarray:
    """Sphere radii [n_dof][per_link]; centres are placed by the callers along
    each link's child-origin vector."""
    rng = np.random.default_rng(seed)
    return rng.uniform(r_lo, r_hi, size=(n_dof, per_link))


# Workload definitions (sizes and generator seeds) of the IK configurations.
IK_PARITY = dict(name="ik7_parity_256x1", robot_seed=100, n_dof=7, batch=256, n_seeds=1,
                 target_seed=200, seed_seed=300, max_iters=30, early_exit=0)
IK_THROUGHPUT = dict(name="ik7_throughput_65536x8", robot_seed=100, n_dof=7, batch=65536, n_seeds=8,
                     target_seed=201, seed_seed=301, max_iters=50, early_exit=1)


def ik_workload(cfg: dict, batch: int | None = None):
    """(robot spec, target configurations [B][n], seeds [B][S][n]) of an IK workload.
    ``batch`` takes the first rows of the full workload."""
    spec = chain_robot(cfg["robot_seed"], cfg["n_dof"])
    B = cfg["batch"]
    qt = uniform_q(cfg["target_seed"], B, spec.dof_lower, spec.dof_upper)
    sd = uniform_q(cfg["seed_seed"], (B, cfg["n_seeds"]), spec.dof_lower, spec.dof_upper)
    if batch is not None:
        qt, sd = qt[:batch], sd[:batch]
    return spec, qt, sd


TRAJOPT = dict(name="trajopt7_1024xT64", robot_seed=100, n_dof=7, batch=1024, T=64, start_seed=600,
               goal_seed=603, obstacle_seed=601, n_obstacles=32, sphere_seed=602, spheres_per_link=4,
               plane=(0.0, 0.0, 1.0, -0.15), reach=(0.5, 1.6), iters=50, candidates=16)


def sphere_obstacles_shell(seed: int, count: int, r_in: float, r_out: float, z_min: float,
                           r_lo=0.05, r_hi=0.2) -> np.ndarray:
    """Obstacle spheres [count][4]: centres uniform in the shell r_in <= |c| <= r_out
    above z_min, radii uniform in [r_lo, r_hi]."""
    rng = np.random.default_rng(seed)
    out = np.zeros((count, 4))
    i = 0
    while i < count:
        c = rng.uniform(-r_out, r_out, 3)
        if not (r_in <= np.linalg.norm(c) <= r_out) or c[2] < z_min:
            continue
        out[i, :3] = c
        out[i, 3] = rng.uniform(r_lo, r_hi)
        i += 1
    return out


# Mobile-base IK: reachable poses of the 7-DoF chain from the fixed base,
# shifted by a planar translation uniform in [-shift, shift]^2 (z unchanged).
MOBILE = dict(name="mobile_ik7_16384x8", robot_seed=100, n_dof=7, batch=16384, n_seeds=8, target_seed=800,
              shift_seed=801, seed_seed=802, shift=1.0, max_iters=50, tol_pos=5e-3, tol_rot=0.05)


def mobile_workload(cfg: dict = MOBILE, batch: int | None = None):
    """(arm spec, mobile spec, arm configurations of the reachable poses [B][n],
    planar shifts [B][2], arm seeds [B][S][n]).  Targets are the arm's FK of
    the configurations with the shift added to the translation; base seeds
    start at the origin (x = y = theta = 0)."""
    arm = chain_robot(cfg["robot_seed"], cfg["n_dof"])
    B = cfg["batch"] if batch is None else batch
    qt = uniform_q(cfg["target_seed"], B, arm.dof_lower, arm.dof_upper)
    rng = np.random.default_rng(cfg["shift_seed"])
    shift = rng.uniform(-cfg["shift"], cfg["shift"], size=(B, 2))
    sd = uniform_q(cfg["seed_seed"], (B, cfg["n_seeds"]), arm.dof_lower, arm.dof_upper)
    return arm, mobile_base_robot(arm), qt, shift, sd


def trajopt_workload(cfg: dict, batch: int | None = None):
    """(robot spec, candidate start configs [C*B][n], candidate goal configs [C*B][n],
    link sphere radii [n][S], obstacles [n_obs][4], plane [4]) with C = cfg['candidates'].
    Callers keep the first B candidates that clear the scene (by their own forward
    kinematics) and take goal poses as FK of the goal configurations."""
    spec = chain_robot(cfg["robot_seed"], cfg["n_dof"])
    B = cfg["batch"] if batch is None else batch
    C = cfg["candidates"] * cfg["batch"]
    qs = uniform_q(cfg["start_seed"], C, spec.dof_lower, spec.dof_upper)
    qg = uniform_q(cfg["goal_seed"], C, spec.dof_lower, spec.dof_upper)
    radii = link_spheres(cfg["sphere_seed"], cfg["n_dof"], cfg["spheres_per_link"])
    plane = np.asarray(cfg["plane"], np.float64)
    obs = sphere_obstacles_shell(cfg["obstacle_seed"], cfg["n_obstacles"], cfg["reach"][0], cfg["reach"][1],
                                 plane[3])
    return spec, qs, qg, radii, obs, plane


def linear_interpolation(q0, q1, T):
    """[B][T][n] straight line from q0 [B][n] to q1 [B][n] in joint space."""
    s = np.linspace(0.0, 1.0, T)[None, :, None]
    return (1.0 - s) * np.asarray(q0)[:, None, :] + s * np.asarray(q1)[:, None, :]


UNEVEN = dict(name="uneven_6_7_24_30", batch_seed=400, batch_lo=1, batch_hi=4096, n_seeds=8, target_seed=410,
              seed_seed=420, max_iters=50)


def uneven_workload(cfg: dict = UNEVEN, scale: float = 1.0):
    """The four robots of the uneven batch with their target frames, target kinds,
    per-robot batch sizes (uniform in [batch_lo, batch_hi], times `scale`), target
    configurations and seeds: [(name, spec, links, kinds, q_targets [B][n], seeds [B][S][n])]."""
    sizes = batch_sizes(cfg["batch_seed"], 4, cfg["batch_lo"], cfg["batch_hi"])
    hand, tips = hand_robot(102)
    hum, ends = humanoid_robot(103)
    c6, c7 = chain_robot(101, 6), chain_robot(100, 7)
    robots = [("chain6", c6, [len(c6["parent"]) - 1], None),
              ("chain7", c7, [len(c7["parent"]) - 1], None),
              ("hand24", hand, list(tips), [TARGET_POSITION] * len(tips)),
              ("humanoid30", hum, list(ends), None)]
    out = []
    for i, (name, spec, links, kinds) in enumerate(robots):
        B = max(1, int(round(sizes[i] * scale)))
        qt = uniform_q(cfg["target_seed"] + i, B, spec.dof_lower, spec.dof_upper)
        sd = uniform_q(cfg["seed_seed"] + i, (B, cfg["n_seeds"]), spec.dof_lower, spec.dof_upper)
        out.append((name, spec, links, kinds, qt, sd))
    return out
