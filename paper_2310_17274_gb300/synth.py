"""Seeded synthetic inputs: robot chain + sphere model, box worlds, problems.

This module holds none of the method's arithmetic (no kinematics, no distance,
no cost).  Where an input depends on the method -- a reachable goal pose is
the forward kinematics of a sampled configuration, and a world keeps only boxes
that do not touch the start configuration -- the caller passes that step in as
a function (``goal_fn``, ``reject_box``).  Tests pass the oracle's; the bench
passes the library's.  Both sides of a parity test therefore read the very same
arrays.

Shapes follow the paper's workloads (7 DOF, about 60 spheres, 32-48 timesteps,
tens of seeds; App. B "cuRobo Parameters"), since its Franka model and its
problem datasets are not available:

* robot (seed 0): F_j = Rot_x(psi_j) Trans(0, 0, l_j), l_j ~ U[0.1, 0.35],
  psi_j ~ U[-0.5, 0.5] (psi_0 = 0), F_ee = Trans(0, 0, l_ee); axes z, y, z, y,
  z, y, z; limits +-2.8 (z joints) / +-1.7 (y joints) rad, velocity 2 rad/s,
  acceleration 15 rad/s^2, jerk 500 rad/s^3; spheres per link 6 (M = 42) or
  9, 9, 9, 9, 8, 8, 8 (M = 60) with centres (U[-.04,.04], U[-.04,.04],
  U[0, l_next]) and radii U[0.03, 0.08]; self-collision pair set = pairs of
  spheres on links at least two apart (consecutive links excluded, Sec. 3.2).
* world: half extents U[0.05, 0.3]^3, centres U[-0.8, 0.8]^3, yaw U[-pi, pi].
* problem: q_start, q_goal ~ U(limits); goal = FK(q_goal) via ``goal_fn``;
  seed b = linear interpolation q_start -> clip(q_goal + eps_b) over H steps,
  eps_0 = 0, eps_b ~ N(0, 0.3^2); IK seeds ~ U(limits).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

AXES_7 = (2, 1, 2, 1, 2, 1, 2)
SPHERES_42 = (6, 6, 6, 6, 6, 6, 6)
SPHERES_60 = (9, 9, 9, 9, 8, 8, 8)


@dataclass
class Robot:
    fixed_tf: np.ndarray     # [dof+1, 12] row-major 3x4: F_0..F_{dof-1}, F_ee
    axis: np.ndarray         # [dof] int32, 0 = x, 1 = y, 2 = z
    q_lo: np.ndarray         # [dof]
    q_hi: np.ndarray
    v_max: np.ndarray
    a_max: np.ndarray
    j_max: np.ndarray
    spheres: np.ndarray      # [M, 4] centre in link frame, radius
    sphere_link: np.ndarray  # [M] int32
    pairs: np.ndarray        # [P, 2] int32

    @property
    def dof(self) -> int:
        return int(len(self.axis))

    @property
    def n_spheres(self) -> int:
        return int(len(self.spheres))

    @property
    def n_pairs(self) -> int:
        return int(len(self.pairs))


@dataclass
class World:
    pose: np.ndarray         # [K, 7] centre xyz, quaternion wxyz
    half_ext: np.ndarray     # [K, 3]

    @property
    def n(self) -> int:
        return int(len(self.pose))


@dataclass
class Problem:
    world: World
    q_start: np.ndarray      # [dof]
    goal: np.ndarray         # [7] xyz + quaternion wxyz
    seeds: np.ndarray        # [B, H, dof]
    q_goal: Optional[np.ndarray] = None

    @property
    def n_seeds(self) -> int:
        return int(self.seeds.shape[0])

    @property
    def horizon(self) -> int:
        return int(self.seeds.shape[1])


def _rot_x(psi):
    c, s = np.cos(psi), np.sin(psi)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _tf(R, p):
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = p
    return T.reshape(12)


def make_robot(spheres_per_link=SPHERES_60, seed: int = 0, pair_min_link_gap: int = 2,
               axes=AXES_7) -> Robot:
    rng = np.random.default_rng(seed)
    dof = len(axes)
    lengths = rng.uniform(0.1, 0.35, size=dof + 1)           # l_0..l_{dof-1}, l_ee
    psi = rng.uniform(-0.5, 0.5, size=dof)
    psi[0] = 0.0
    F = np.zeros((dof + 1, 12))
    for j in range(dof):
        R = _rot_x(psi[j])
        F[j] = _tf(R, R @ np.array([0.0, 0.0, lengths[j]]))
    F[dof] = _tf(np.eye(3), np.array([0.0, 0.0, lengths[dof]]))
    axis = np.asarray(axes, dtype=np.int32)
    q_lim = np.where(axis == 2, 2.8, 1.7)
    spheres, link = [], []
    for l, n in enumerate(spheres_per_link):
        l_next = lengths[l + 1]
        for _ in range(n):
            c = [rng.uniform(-0.04, 0.04), rng.uniform(-0.04, 0.04), rng.uniform(0.0, l_next)]
            spheres.append(c + [rng.uniform(0.03, 0.08)])
            link.append(l)
    spheres = np.asarray(spheres)
    link = np.asarray(link, dtype=np.int32)
    pairs = [(i, j) for i in range(len(link)) for j in range(i + 1, len(link))
             if abs(int(link[i]) - int(link[j])) >= pair_min_link_gap]
    return Robot(fixed_tf=F, axis=axis, q_lo=-q_lim, q_hi=q_lim.copy(),
                 v_max=np.full(dof, 2.0), a_max=np.full(dof, 15.0), j_max=np.full(dof, 500.0),
                 spheres=spheres, sphere_link=link,
                 pairs=np.asarray(pairs, dtype=np.int32).reshape(-1, 2))


def _random_box(rng):
    he = rng.uniform(0.05, 0.3, size=3)
    c = rng.uniform(-0.8, 0.8, size=3)
    yaw = rng.uniform(-np.pi, np.pi)
    return np.concatenate([c, [np.cos(yaw / 2), 0.0, 0.0, np.sin(yaw / 2)]]), he


def make_world(n_boxes: int, seed: int,
               reject_box: Optional[Callable[[np.ndarray, np.ndarray], bool]] = None,
               max_tries: int = 200) -> World:
    """n_boxes random cuboids; a box for which reject_box(pose7, half_ext) is
    true is drawn again (up to max_tries times, then kept)."""
    rng = np.random.default_rng(seed)
    pose = np.zeros((n_boxes, 7))
    he = np.zeros((n_boxes, 3))
    for k in range(n_boxes):
        for _ in range(max_tries):
            p, h = _random_box(rng)
            if reject_box is None or not reject_box(p, h):
                break
        pose[k], he[k] = p, h
    return World(pose=pose, half_ext=he)


def uniform_config(rng, robot: Robot, n=None):
    size = (robot.dof,) if n is None else (n, robot.dof)
    return rng.uniform(robot.q_lo, robot.q_hi, size=size)


def linear_seeds(rng, robot: Robot, q_start, q_goal, n_seeds: int, horizon: int, noise=0.3):
    """seed b(t) = q_start + (t/H) (clip(q_goal + eps_b) - q_start), t = 1..H."""
    eps = rng.normal(0.0, noise, size=(n_seeds, robot.dof))
    eps[0] = 0.0
    ends = np.clip(q_goal[None, :] + eps, robot.q_lo, robot.q_hi)
    w = (np.arange(1, horizon + 1) / horizon)[None, :, None]
    return q_start[None, None, :] + w * (ends[:, None, :] - q_start[None, None, :])


def make_problem(robot: Robot, world: World, seed: int, n_seeds: int, horizon: int,
                 goal_fn: Callable[[np.ndarray], np.ndarray],
                 q_start: Optional[np.ndarray] = None) -> Problem:
    rng = np.random.default_rng(seed)
    qs = uniform_config(rng, robot) if q_start is None else np.asarray(q_start, dtype=np.float64)
    qg = uniform_config(rng, robot)
    seeds = linear_seeds(rng, robot, qs, qg, n_seeds, horizon)
    return Problem(world=world, q_start=qs, goal=np.asarray(goal_fn(qg), dtype=np.float64),
                   seeds=seeds, q_goal=qg)


def make_ik_problems(robot: Robot, world: World, seed: int, n_goals: int, n_seeds: int,
                     goal_fn: Callable[[np.ndarray], np.ndarray]):
    """n_goals IK problems (H = 1): goals from configurations sampled within
    the limits, seeds sampled within the limits."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_goals):
        qg = uniform_config(rng, robot)
        seeds = uniform_config(rng, robot, n_seeds)[:, None, :]
        qs = uniform_config(rng, robot)
        out.append(Problem(world=world, q_start=qs, goal=np.asarray(goal_fn(qg)), seeds=seeds,
                           q_goal=qg))
    return out


@dataclass
class Config:
    name: str
    spheres_per_link: tuple
    n_boxes: int
    n_seeds: int
    horizon: int
    iters: int
    alphas: tuple
    world_seed: int
    extra: dict = field(default_factory=dict)


ALPHA_4 = (0.01, 0.3, 0.7, 1.0)
ALPHA_8 = (0.01, 0.1, 0.2, 0.3, 0.5, 0.7, 0.9, 1.0)

# The five workloads: tiny, trajectory optimisation, batched IK, uneven batch, serving.
CONFIGS = {
    "tiny": Config("tiny", SPHERES_42, 8, 4, 32, 25, ALPHA_4, 1),
    "trajopt": Config("trajopt", SPHERES_60, 32, 32, 48, 100, ALPHA_8, 2),
    "ik": Config("ik", SPHERES_60, 40, 32, 1, 50, ALPHA_4, 3, dict(n_goals=1000)),
    "uneven": Config("uneven", SPHERES_60, 0, 0, 0, 100, ALPHA_4, 4, dict(n_problems=64)),
    "serve": Config("serve", SPHERES_60, 0, 32, 48, 100, ALPHA_8, 5, dict(rate=500.0)),
}


def uneven_shapes(seed: int = 4, n_problems: int = 64):
    """(n_boxes, n_seeds, horizon) per problem of the uneven batch: boxes
    log-uniform in [5, 200], seeds in {4, 16, 32, 64}, horizons in {32, 48, 64}."""
    rng = np.random.default_rng(seed)
    K = np.rint(np.exp(rng.uniform(np.log(5), np.log(200), size=n_problems))).astype(int)
    B = rng.choice([4, 16, 32, 64], size=n_problems)
    H = rng.choice([32, 48, 64], size=n_problems)
    return [(int(k), int(b), int(h)) for k, b, h in zip(K, B, H)]
