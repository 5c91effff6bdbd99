"""Construction of the synthetic trajectory-optimisation scenes (not the
optimiser): candidate start and goal configurations are kept only if every
link sphere clears every obstacle and the ground plane by the margin, so that
each problem has collision-free endpoints.  Callers pass the joint-frame
positions from their own forward kinematics."""
from __future__ import annotations

import numpy as np


def sphere_centres(points: np.ndarray, S: int) -> np.ndarray:
    """points [B][n+1][3] (joint origins then the tool point) -> centres [B][n][S][3]
    at p_j + (s + 1/2)/S (p_{j+1} - p_j)."""
    a = (np.arange(S) + 0.5) / S
    p0, p1 = points[:, :-1, None, :], points[:, 1:, None, :]
    return p0 + a[None, None, :, None] * (p1 - p0)


def clearance(points: np.ndarray, radii: np.ndarray, obstacles: np.ndarray, plane: np.ndarray) -> np.ndarray:
    """Smallest signed sphere distance per configuration [B] (the first link is not
    tested against the plane)."""
    c = sphere_centres(points, radii.shape[1])
    d = np.full(points.shape[0], np.inf)
    if len(obstacles):
        v = c[:, :, :, None, :] - obstacles[None, None, None, :, :3]
        dd = np.linalg.norm(v, axis=-1) - radii[None, :, :, None] - obstacles[None, None, None, :, 3]
        d = np.minimum(d, dd.reshape(len(d), -1).min(axis=1))
    dp = c[:, 1:] @ plane[:3] - plane[3] - radii[None, 1:]
    return np.minimum(d, dp.reshape(len(d), -1).min(axis=1))


def pick_clear(q: np.ndarray, points: np.ndarray, radii, obstacles, plane, margin: float, count: int):
    """The first `count` configurations whose clearance exceeds `margin`."""
    ok = np.nonzero(clearance(points, radii, obstacles, plane) > margin)[0]
    if len(ok) < count:
        raise ValueError(f"only {len(ok)} of {len(q)} candidates clear the scene; need {count}")
    return q[ok[:count]]
