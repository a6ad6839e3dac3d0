"""Seeded scenes shared by the parity tests: synth inputs, with the oracle as
the goal / rejection function, so both sides read identical arrays."""
import numpy as np

import oracle
from paper_2310_17274_gb300 import synth


def f32(a):
    """Round to float32 and back: the exact values the GPU path receives."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def as_f32_world(w):
    return synth.World(pose=f32(w.pose), half_ext=f32(w.half_ext))


def as_f32_robot(rb):
    return synth.Robot(fixed_tf=f32(rb.fixed_tf), axis=rb.axis, q_lo=f32(rb.q_lo), q_hi=f32(rb.q_hi),
                       v_max=f32(rb.v_max), a_max=f32(rb.a_max), j_max=f32(rb.j_max),
                       spheres=f32(rb.spheres), sphere_link=rb.sphere_link, pairs=rb.pairs)


def scene(spheres=synth.SPHERES_42, n_boxes=8, n_seeds=4, horizon=32, world_seed=1,
          problem_seed=7, robot_seed=0):
    rb = as_f32_robot(synth.make_robot(spheres, seed=robot_seed))
    rng = np.random.default_rng(problem_seed + 1000)
    qs = f32(synth.uniform_config(rng, rb))
    w = as_f32_world(synth.make_world(n_boxes, world_seed,
                                      lambda p, h: oracle.start_collides_with_box(rb, qs, p, h)))
    pr = synth.make_problem(rb, w, problem_seed, n_seeds, horizon,
                            lambda q: oracle.goal_pose_from_fk(rb, q), q_start=qs)
    pr.goal = f32(pr.goal)
    pr.seeds = f32(pr.seeds)
    return rb, w, pr


def line_search_batch(pr, rng, alphas=(0.01, 0.3, 0.7, 1.0), scale=0.2):
    """Seeds x step sizes around each seed, like one batch of line-search
    candidates: [B * n_alpha, H, dof]."""
    B, H, D = pr.seeds.shape
    d = rng.normal(0, scale, size=(B, H, D))
    out = np.stack([pr.seeds + a * d for a in alphas], axis=1).reshape(B * len(alphas), H, D)
    return f32(out)
