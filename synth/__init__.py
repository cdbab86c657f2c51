"""Seeded synthetic correspondence sets for the registration workloads.

This module only draws inputs: point clouds, a ground-truth rigid transform,
inlier noise and uniform outliers.  It contains none of the registration
method's arithmetic (no compatibility test, no SC^2, no clique search, no
Kabsch, no inlier count), so both the FP64 CPU oracle and the CUDA path can
consume its output without sharing any code.

Every draw comes from ``numpy.random.Generator(PCG64(seed))`` in a fixed
order, so a (shape, n, inlier ratio, seed) tuple always yields the same
float32 arrays on any machine with NumPy >= 1.17.

Problem model (Sec. 3.1 and App. A.1 of the paper): correspondences
m_i = (x_i, y_i) with y_i = T(x_i) + r_i.  For inliers r_i ~ N(0, sigma^2 I);
outliers have y_i drawn uniformly in the axis-aligned bounding box of the
transformed source cloud, independent of x_i.

The paper measures on 3DMatch / 3DLoMatch / KITTI correspondences, which are
not available here; the "indoor" shape stands in for room-scale scans and
the "outdoor" shape for street-scale scans.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "SHAPES",
    "make_problem",
    "make_batch",
    "rotation_error_deg",
    "translation_error",
]


@dataclass(frozen=True)
class Shape:
    """Value distributions and thresholds of one workload family."""

    name: str
    box_lo: tuple
    box_hi: tuple
    rot: str              # "so3" (uniform on SO(3)) or "yaw_rp" (yaw + small roll/pitch)
    t_lo: tuple
    t_hi: tuple
    sigma: float          # inlier noise, metres per axis
    tau: float            # compatibility threshold (Eq. 1)
    theta: float          # inlier threshold for the inlier number (Sec. 3.5)
    k1: int               # pivots
    re_deg: float         # success: rotation error below this
    te_m: float           # success: translation error below this


SHAPES = {
    # N=1000 cube [0,3]^3, 10% inliers (small parity case)
    "cube": Shape("cube", (0.0, 0.0, 0.0), (3.0, 3.0, 3.0), "so3",
                  (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0),
                  0.01, 0.1, 0.1, 1000, 15.0, 0.3),
    # room-scale: [0,4]x[0,4]x[0,3] m, 3DMatch-like thresholds
    "indoor": Shape("indoor", (0.0, 0.0, 0.0), (4.0, 4.0, 3.0), "so3",
                    (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0),
                    0.01, 0.1, 0.1, 2000, 15.0, 0.3),
    # street-scale: [-35,35]^2 x [-2,3] m, KITTI-like thresholds
    "outdoor": Shape("outdoor", (-35.0, -35.0, -2.0), (35.0, 35.0, 3.0), "yaw_rp",
                     (-5.0, -5.0, -0.5), (5.0, 5.0, 0.5),
                     0.05, 0.6, 0.6, 1000, 5.0, 0.6),
}


@dataclass
class Problem:
    x: np.ndarray          # float32 [n,3] source keypoints
    y: np.ndarray          # float32 [n,3] target keypoints
    R_gt: np.ndarray       # float64 [3,3], y = R_gt x + t_gt for inliers
    t_gt: np.ndarray       # float64 [3]
    inlier: np.ndarray     # bool [n]
    tau: float
    theta: float
    k1: int
    re_deg: float
    te_m: float
    shape: str
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def _quat_to_rot(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _uniform_so3(rng):
    # Shoemake's subgroup algorithm: a uniform unit quaternion from 3 uniforms.
    u1, u2, u3 = rng.random(3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    q = (b * math.cos(2 * math.pi * u3), a * math.sin(2 * math.pi * u2),
         a * math.cos(2 * math.pi * u2), b * math.sin(2 * math.pi * u3))
    return _quat_to_rot(q)


def _yaw_roll_pitch(rng):
    yaw = rng.uniform(-math.pi, math.pi)
    pitch, roll = np.deg2rad(rng.uniform(-5.0, 5.0, 2))
    cz, sz = math.cos(yaw), math.sin(yaw)
    cy, sy = math.cos(pitch), math.sin(pitch)
    cx, sx = math.cos(roll), math.sin(roll)
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1.0]])
    Ry = np.array([[cy, 0, sy], [0, 1.0, 0], [-sy, 0, cy]])
    Rx = np.array([[1.0, 0, 0], [0, cx, -sx], [0, sx, cx]])
    return Rz @ Ry @ Rx


def make_problem(shape: str, n: int, inlier_ratio: float, seed: int, *,
                 sigma: float | None = None, k1: int | None = None,
                 tau: float | None = None, theta: float | None = None) -> Problem:
    """Draw one seeded correspondence set of the given workload shape."""
    sh = SHAPES[shape]
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(sh.box_lo, sh.box_hi, size=(n, 3))
    R = _uniform_so3(rng) if sh.rot == "so3" else _yaw_roll_pitch(rng)
    t = rng.uniform(sh.t_lo, sh.t_hi)
    n_in = int(round(inlier_ratio * n))
    perm = rng.permutation(n)
    inl = np.zeros(n, dtype=bool)
    inl[perm[:n_in]] = True
    yt = x @ R.T + t
    s = sh.sigma if sigma is None else sigma
    y = np.empty_like(yt)
    noise = rng.normal(0.0, 1.0, size=(n_in, 3)) * s
    y[perm[:n_in]] = yt[perm[:n_in]] + noise
    lo, hi = yt.min(axis=0), yt.max(axis=0)
    y[perm[n_in:]] = rng.uniform(lo, hi, size=(n - n_in, 3))
    return Problem(
        x=np.ascontiguousarray(x, dtype=np.float32),
        y=np.ascontiguousarray(y, dtype=np.float32),
        R_gt=R, t_gt=t, inlier=inl,
        tau=sh.tau if tau is None else tau,
        theta=sh.theta if theta is None else theta,
        k1=sh.k1 if k1 is None else k1,
        re_deg=sh.re_deg, te_m=sh.te_m, shape=shape, seed=seed,
        meta={"inlier_ratio": inlier_ratio, "sigma": s},
    )


def make_batch(num: int, seed: int, n_lo: int = 500, n_hi: int = 5000,
               ratio_lo: float = 0.02, ratio_hi: float = 0.20):
    """A list of independent problems of uneven size (batched workload).

    Each problem is indoor- or outdoor-shaped with probability 0.5, N uniform
    in [n_lo, n_hi] and inlier ratio uniform in [ratio_lo, ratio_hi].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for p in range(num):
        shape = "indoor" if rng.random() < 0.5 else "outdoor"
        n = int(rng.integers(n_lo, n_hi + 1))
        ratio = float(rng.uniform(ratio_lo, ratio_hi))
        out.append(make_problem(shape, n, ratio, seed * 100003 + p))
    return out


def rotation_error_deg(R_gt, R) -> float:
    """RE = arccos((tr(R_gt^T R) - 1) / 2) in degrees (success metric, Sec. 4.1)."""
    c = (np.trace(np.asarray(R_gt, dtype=np.float64).T @ np.asarray(R, dtype=np.float64)) - 1.0) / 2.0
    return float(np.degrees(np.arccos(np.clip(c, -1.0, 1.0))))


def translation_error(t_gt, t) -> float:
    """TE = ||t_gt - t||_2 in metres (success metric, Sec. 4.1)."""
    return float(np.linalg.norm(np.asarray(t_gt, dtype=np.float64) - np.asarray(t, dtype=np.float64)))
