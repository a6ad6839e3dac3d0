"""The batched, graph-captured solve (cr_solve) against the step entry points,
against itself in other launch forms, against the oracle (distributionally:
end-to-end optimised trajectories are chaotic and parity there is unpinned)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_17274_gb300 import crgb, synth

from scenes import f32, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2310_17274_gb300 import build
    build.build_library()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def ctx():
    return crgb.Context(0)


def _spec(W, pr):
    return crgb.ProblemSpec(W, pr.q_start, pr.goal, pr.seeds.shape[1], seeds=pr.seeds)


def _stepwise(R, W, pr, params, iters):
    """The same iterations through cr_eval / cr_opt_propose / cr_opt_select."""
    P = crgb.make_params(params)
    B, H, D = pr.seeds.shape
    na = P.n_alpha
    st = crgb.OptBuffers(B, H, D, P.history, na)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H)
    x = torch.tensor(pr.seeds, dtype=torch.float32, device="cuda")
    out = crgb.evaluate(R, spec, x, P)
    st.x.copy_(x.view(B, -1))
    st.g.copy_(out["grad"].view(B, -1))
    st.c.copy_(out["cost"])
    st.best_x.copy_(st.x)
    st.best_c.copy_(st.c)
    st.best_cfree.copy_(out["cfree"])
    for it in range(iters):
        crgb.opt_propose(R, P, st)
        ev = crgb.evaluate(R, spec, st.cand.view(B * na, H, D), P)
        st.cand_cost.copy_(ev["cost"].view(B, na))
        st.cand_grad.copy_(ev["grad"].view(B, na, -1))
        st.cand_cfree.copy_(ev["cfree"].view(B, na))
        crgb.opt_select(R, P, st)
    torch.cuda.synchronize()
    return st


def test_solve_equals_step_entry_points(ctx):
    rb, w, pr = scene(n_seeds=4, horizon=32)
    R, W = crgb.Robot(rb), crgb.World(w)
    for graph, persistent in [(False, False), (True, True)]:
        out = crgb.solve(ctx, R, [_spec(W, pr)], None, iters=6, graph=graph, persistent=persistent)[0]
        torch.cuda.synchronize()
        st = _stepwise(R, W, pr, None, 6)
        assert torch.equal(out.traj.view(4, -1), st.best_x)
        assert torch.equal(out.cost, st.best_c)
        assert torch.equal(out.cfree, st.best_cfree)


def test_solve_launch_forms_agree_and_graph_replays(ctx):
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=32, n_seeds=8, horizon=48, world_seed=2)
    R, W = crgb.Robot(rb), crgb.World(w)
    p = dict(alpha=list(synth.ALPHA_8))
    outs = []
    for graph, persistent in [(False, False), (False, True), (True, False), (True, True), (True, True)]:
        o = crgb.solve(ctx, R, [_spec(W, pr)], p, iters=10, graph=graph, persistent=persistent)[0]
        torch.cuda.synchronize()
        outs.append(o)
    for o in outs[1:]:
        assert torch.equal(o.traj, outs[0].traj)
        assert torch.equal(o.cost, outs[0].cost)
        assert torch.equal(o.best, outs[0].best)
    # the replayed graph picks up new problem data with the same shapes
    pr2 = synth.Problem(world=w, q_start=pr.q_start, goal=pr.goal, seeds=f32(pr.seeds[::-1].copy()))
    o2 = crgb.solve(ctx, R, [_spec(W, pr2)], p, iters=10, graph=True, persistent=True)[0]
    torch.cuda.synchronize()
    assert torch.equal(o2.cost, outs[0].cost.flip(0))


def test_batched_problems_equal_alone(ctx):
    """Uneven problems solved together give exactly what each gives alone."""
    rb = scene(spheres=synth.SPHERES_60)[0]
    R = crgb.Robot(rb)
    specs, worlds, probs = [], [], []
    for k, (K, B, H) in enumerate([(5, 4, 32), (40, 16, 48), (12, 4, 64), (0, 2, 32)]):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=K, n_seeds=B, horizon=H, world_seed=10 + k,
                         problem_seed=20 + k)
        W = crgb.World(w)
        worlds.append(W)
        probs.append(pr)
        specs.append(_spec(W, pr))
    together = crgb.solve(ctx, R, specs, None, iters=5, graph=True, persistent=True)
    torch.cuda.synchronize()
    for s, t in zip(specs, together):
        alone = crgb.solve(ctx, R, [s], None, iters=5, graph=False, persistent=False)[0]
        torch.cuda.synchronize()
        assert torch.equal(alone.traj, t.traj)
        assert torch.equal(alone.cost, t.cost)
        assert torch.equal(alone.cfree, t.cfree)
        assert torch.equal(alone.best, t.best)


@pytest.mark.parametrize("flags", [0, None])
def test_small_seeds_equal_wide_kernel(ctx, flags):
    """Seeds of at most 32 variables run one per thread; alone they must give
    bit for bit what the block-wide optimiser gives them inside a batch with a
    long-horizon problem (every dot product in the same order).  Trajectory
    mode with H = 4 (28 variables) and IK mode (7 variables, plus H = 48
    states evaluated as independent states in the same batch)."""
    rb = scene(spheres=synth.SPHERES_60)[0]
    R = crgb.Robot(rb)
    params = None if flags is None else dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE)
    small_h = 4 if flags is None else 1
    specs = []
    for k, (K, B, H) in enumerate([(6, 8, small_h), (12, 4, 48)]):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=K, n_seeds=B, horizon=H, world_seed=30 + k,
                         problem_seed=40 + k)
        specs.append(_spec(crgb.World(w), pr))
    together = crgb.solve(ctx, R, specs, params, iters=6, graph=True, persistent=True)
    torch.cuda.synchronize()
    alone = crgb.solve(ctx, R, [specs[0]], params, iters=6, graph=False, persistent=False)[0]
    torch.cuda.synchronize()
    t = together[0]
    assert torch.equal(alone.traj, t.traj)
    assert torch.equal(alone.cost, t.cost)
    assert torch.equal(alone.cfree, t.cfree)
    assert torch.equal(alone.best, t.best)


def test_ik_small_and_large_batches_agree(ctx):
    """IK solves: alone, a problem of 8 seeds runs the one-warp optimiser and
    the split evaluation; inside a batch of 4104 seeds the per-thread
    optimiser and the one-thread evaluation.  Same bits."""
    rb = scene(spheres=synth.SPHERES_60)[0]
    R = crgb.Robot(rb)
    params = dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE)
    specs = []
    for k, B in enumerate((8, 4096)):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=20, n_seeds=B, horizon=1, world_seed=50 + k,
                         problem_seed=60 + k)
        specs.append(_spec(crgb.World(w), pr))
    together = crgb.solve(ctx, R, specs, params, iters=8, graph=True, persistent=True)
    torch.cuda.synchronize()
    alone = crgb.solve(ctx, R, [specs[0]], params, iters=8, graph=False, persistent=False)[0]
    torch.cuda.synchronize()
    t = together[0]
    assert torch.equal(alone.traj, t.traj)
    assert torch.equal(alone.cost, t.cost)
    assert torch.equal(alone.cfree, t.cfree)
    assert torch.equal(alone.best, t.best)


def test_short_horizon_many_seeds_agree(ctx):
    """Trajectories of 4 states (28 variables): alone, 8 seeds run one warp
    each; inside a batch with 4096 more they run one thread each.  Same bits."""
    rb = scene(spheres=synth.SPHERES_60)[0]
    R = crgb.Robot(rb)
    specs = []
    for k, B in enumerate((8, 4096)):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=10, n_seeds=B, horizon=4, world_seed=70 + k,
                         problem_seed=80 + k)
        specs.append(_spec(crgb.World(w), pr))
    together = crgb.solve(ctx, R, specs, None, iters=6, graph=True, persistent=True)
    torch.cuda.synchronize()
    alone = crgb.solve(ctx, R, [specs[0]], None, iters=6, graph=False, persistent=False)[0]
    torch.cuda.synchronize()
    t = together[0]
    assert torch.equal(alone.traj, t.traj)
    assert torch.equal(alone.cost, t.cost)
    assert torch.equal(alone.best, t.best)


def test_solve_result_is_consistent_with_oracle(ctx):
    """Returned best iterates: their oracle cost matches the reported cost
    (1e-4 rel, unless near a decision threshold) and the reported best index
    is the lowest-cost collision-free seed."""
    rb, w, pr = scene(n_seeds=8, horizon=32, problem_seed=3)
    R, W = crgb.Robot(rb), crgb.World(w)
    out = crgb.solve(ctx, R, [_spec(W, pr)], None, iters=25)[0]
    torch.cuda.synchronize()
    x = f32(out.traj.cpu().numpy())
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, x)
    c = out.cost.cpu().numpy()
    for b in range(8):
        if ref["margin"][b] >= 1e-5:
            assert abs(c[b] - ref["cost"][b]) <= 1e-4 * max(abs(ref["cost"][b]), 1e-2)
            assert bool(out.cfree[b]) == bool(ref["cfree"][b])
    cf = out.cfree.cpu().numpy().astype(bool)
    best = int(out.best)
    if cf.any():
        assert cf[best] and c[best] == c[cf].min()
    else:
        assert c[best] == c.min()
    init = oracle.evaluate(rb, w, pr.q_start, pr.goal, pr.seeds)["cost"]
    assert np.all(c <= init * (1 + 1e-4))


def test_solve_distribution_matches_oracle_tiny(ctx):
    """Tiny workload, 25 iterations: final best-cost quantiles of the GPU
    solve and of the oracle solve agree within 5% (distributional check)."""
    rb, w, pr = scene(n_seeds=16, horizon=32, problem_seed=5)
    R, W = crgb.Robot(rb), crgb.World(w)
    out = crgb.solve(ctx, R, [_spec(W, pr)], None, iters=25)[0]
    torch.cuda.synchronize()
    g = np.sort(out.cost.cpu().numpy())
    o = np.sort(oracle.solve(rb, w, pr.q_start, pr.goal, pr.seeds, 25)["cost"])
    for q in (0.25, 0.5, 0.75):
        a, b = np.quantile(g, q), np.quantile(o, q)
        assert abs(a - b) <= 0.05 * abs(b), (q, a, b)


def test_ik_batch(ctx):
    """Batched collision-free IK (H = 1): many goals in one solve, goals from
    collision-free configurations; solutions verified with the oracle's
    kinematics and distance."""
    rb, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=40, world_seed=3)
    R, W = crgb.Robot(rb), crgb.World(w)
    p = dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE)
    rng = np.random.default_rng(9)
    free_q = []
    while len(free_q) < 16:
        q = f32(synth.uniform_config(rng, rb))
        if oracle.evaluate(rb, w, q, np.array([0, 0, 0, 1.0, 0, 0, 0]), q[None, None], p)["cfree"][0]:
            free_q.append(q)
    specs, goals = [], []
    for q in free_q:
        goal = f32(oracle.goal_pose_from_fk(rb, q))
        seeds = f32(synth.uniform_config(rng, rb, 32)[:, None, :])
        goals.append(goal)
        specs.append(crgb.ProblemSpec(W, free_q[0], goal, 1, seeds=seeds))
    outs = crgb.solve(ctx, R, specs, p, iters=100)
    torch.cuda.synchronize()
    n_ok = 0
    for goal, o in zip(goals, outs):
        b = int(o.best)
        q = o.traj[b, 0].cpu().numpy().astype(np.float64)
        ev = oracle.evaluate(rb, w, free_q[0], goal, q[None, None], p)
        if ev["margin"][0] >= 1e-5:
            assert bool(o.cfree[b]) == bool(ev["cfree"][0])
            # near a converged pose the cost is steep in the end-effector
            # pose: allow what 1e-6 m / 1e-6 rad of pose error can change
            # (FP32 kinematics through seven chained transforms of unit scale)
            _, _, ee = oracle.fk(rb, q)
            _, dp, dR = oracle.goal_cost(p, ee, goal)
            slack = 1e-6 * (np.linalg.norm(dp) + np.linalg.norm(dR))
            assert abs(float(o.cost[b]) - ev["cost"][0]) <= 1e-4 * max(abs(ev["cost"][0]), 1e-2) + slack
        _, _, ee = oracle.fk(rb, q)
        E = ee.reshape(3, 4)
        pos_err = np.linalg.norm(E[:, 3] - goal[:3])
        if ev["cfree"][0] and pos_err <= 5e-3:
            n_ok += 1
    assert n_ok >= 4, n_ok


def test_tile_shapes_do_not_change_results_and_autotune():
    """The autotuner's choices (CTA size, states per tile for short horizons)
    change speed only: results are bit-identical under every tile shape."""
    ctx = crgb.Context(0)
    rb, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=24, world_seed=4)
    R, W = crgb.Robot(rb), crgb.World(w)
    rng = np.random.default_rng(3)
    specs = []
    for g in range(6):   # IK problems (H = 1) and short trajectories (H = 8)
        H = 1 if g % 2 == 0 else 8
        qs = f32(synth.uniform_config(rng, rb))
        seeds = f32(synth.uniform_config(rng, rb, 12 * H).reshape(12, H, rb.dof))
        goal = f32(oracle.goal_pose_from_fk(rb, synth.uniform_config(rng, rb)))
        specs.append(crgb.ProblemSpec(W, qs, goal, H, seeds=seeds))
    ref = crgb.solve(ctx, R, specs, None, iters=4)
    torch.cuda.synchronize()
    for block, short, nc in [(256, 8, 1), (512, 64, 0), (256, 16, 0), (512, 32, 1)]:
        for H in (1, 8):
            crgb.tune_set(ctx, rb.n_spheres, w.n, H, block, short, nc)
        out = crgb.solve(ctx, R, specs, None, iters=4)
        torch.cuda.synchronize()
        for a, b in zip(ref, out):
            assert torch.equal(a.traj, b.traj) and torch.equal(a.cost, b.cost)
    choice = crgb.autotune(ctx, R, specs, None, iters=2)
    assert choice["block"] in (256, 512) and choice["short_tile"] in (8, 16, 32, 64)
    assert choice["no_cache"] in (0, 1)
    assert choice["ms"] > 0
    out = crgb.solve(ctx, R, specs, None, iters=4)
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert torch.equal(a.traj, b.traj) and torch.equal(a.cost, b.cost)


def test_status_word_reports_non_finite_seeds():
    """The device status word of each problem: CR_ENAN (6) for a problem with
    a NaN in one seed, CR_OK for the problem beside it, whose results are
    those it has alone."""
    rb, w, pr = scene(n_seeds=4, horizon=32)
    R, W = crgb.Robot(rb), crgb.World(w)
    bad = pr.seeds.copy()
    bad[2, 5, 3] = np.nan
    good = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32, seeds=pr.seeds)
    nan = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32, seeds=bad)
    ctx = crgb.Context(0)
    og, on = crgb.solve(ctx, R, [good, nan], iters=5)
    alone = crgb.solve(ctx, R, [good], iters=5)[0]
    torch.cuda.synchronize()
    assert int(og.status) == 0 and int(on.status) == 6
    assert torch.equal(og.traj, alone.traj) and torch.equal(og.cost, alone.cost)
    c = on.cost.cpu().numpy()
    assert not np.isfinite(c[2]) and np.isfinite(c[[0, 1, 3]]).all()
    assert int(on.best) != 2
