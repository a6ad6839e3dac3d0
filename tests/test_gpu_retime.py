"""Retiming (App. "Time-step Discretization") through cr_retime against the
oracle, and the two-stage time-discretised solve of Alg. "Time Discretization"."""
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


def test_retime_matches_oracle():
    rb, w, pr = scene(n_seeds=4, horizon=32, problem_seed=21)
    rng = np.random.default_rng(3)
    theta = f32(np.concatenate([pr.seeds, pr.seeds + rng.normal(0, 0.02, size=pr.seeds.shape),
                                np.tile(pr.q_start, (1, 32, 1))]))
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32)
    dt = crgb.retime(R, spec, torch.tensor(theta, dtype=torch.float32, device="cuda")).cpu().numpy()
    ref = np.array([oracle.retime(rb, pr.q_start, t) for t in theta])
    np.testing.assert_allclose(dt[:-1], ref[:-1], rtol=2e-5)
    assert dt[-1] < 1e-3 and ref[-1] < 1e-3     # a trajectory that never moves


@pytest.mark.parametrize("graph", [True, False])
def test_time_discretized_solve_stages(graph):
    """cr_solve_timeopt (Alg. "Time Discretization", every stage on the
    device) checked stage by stage: the first solve equals cr_solve at the
    coarse step without jerk, bit for bit; dt_opt is the oracle's retiming of
    its best seed; the second solve's weights are the oracle's scaling to
    dt_opt; the second solve equals cr_solve from the first solve's seeds with
    those weights, bit for bit; every seed's step and score match the oracle's
    and the chosen seed is the oracle's choice (unless two scores are within
    FP32 rounding of each other)."""
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=8, n_seeds=8, horizon=32, problem_seed=22)
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32, seeds=pr.seeds)
    ctx = crgb.Context(0)
    out, to = crgb.time_discretized_solve(ctx, R, spec, iters=(20, 20), graph=graph)
    torch.cuda.synchronize()
    st = to.stage.cpu().numpy()
    p1 = dict(dt=float(st[0]), w_vel=float(st[1]), w_acc=float(st[2]), w_jerk=float(st[3]))
    ref1 = oracle.time_scaled_params(None, 0.25, jerk=False)
    for k, v in zip(("dt", "w_vel", "w_acc", "w_jerk"), st[:4]):
        assert v == pytest.approx(ref1[k], rel=1e-6), k
    o1 = crgb.solve(ctx, R, [spec], p1, iters=20, graph=graph)[0]
    torch.cuda.synchronize()
    b1 = int(o1.best)
    assert torch.equal(to.first, o1.traj[b1])
    dt_opt = max(oracle.retime(rb, pr.q_start, o1.traj[b1].cpu().numpy().astype(np.float64)), 1e-3)
    assert st[4] == pytest.approx(dt_opt, rel=2e-5)
    ref2 = oracle.time_scaled_params(None, float(st[4]), jerk=True)
    for k, v in zip(("dt", "w_vel", "w_acc", "w_jerk"), st[4:]):
        assert v == pytest.approx(ref2[k], rel=1e-5), k
    p2 = dict(dt=float(st[4]), w_vel=float(st[5]), w_acc=float(st[6]), w_jerk=float(st[7]))
    o2 = crgb.solve(ctx, R, [spec], p2, iters=20, graph=graph, device_seeds=[o1.traj.contiguous()])[0]
    torch.cuda.synchronize()
    for k in ("traj", "cost", "cfree", "best", "status"):
        assert torch.equal(getattr(out, k), getattr(o2, k)), k
    assert int(out.status) == 0
    traj = out.traj.cpu().numpy().astype(np.float64)
    cf = out.cfree.cpu().numpy().astype(bool)
    dts = to.dt.cpu().numpy()
    ref_dt = np.array([oracle.retime(rb, pr.q_start, t) for t in traj])
    np.testing.assert_allclose(dts, ref_dt, rtol=2e-5)
    score, rbest = oracle.rank_seeds(rb, pr.q_start, pr.goal, traj, cf, dt=f32(dts), w_pose=1.0, w_jerk=1e-3,
                                     w_time=1.0)
    np.testing.assert_allclose(to.score.cpu().numpy(), score, rtol=1e-4, atol=1e-6)
    chosen = int(to.chosen)
    if rbest < 0:
        assert chosen == int(out.best)
    else:
        ok = np.where(cf, score, np.inf)
        second = np.partition(ok, 1)[1] if cf.sum() > 1 else np.inf
        if second - ok[rbest] > 1e-4 * abs(ok[rbest]):
            assert chosen == rbest
        assert cf[chosen]
        # retimed to its own step the chosen trajectory sits at a limit (oracle stencils)
        v, a, j = oracle.stencil(pr.q_start, traj[chosen], float(dts[chosen]))
        ratio = max(np.max(np.abs(v) / rb.v_max), np.max(np.abs(a) / rb.a_max), np.max(np.abs(j) / rb.j_max))
        assert ratio == pytest.approx(1.0, rel=1e-4)


def test_time_discretized_solve_batch_equals_alone():
    """Two problems in one time-discretised solve give what each gives alone."""
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=8, n_seeds=4, horizon=32, problem_seed=23)
    _, w2, pr2 = scene(spheres=synth.SPHERES_60, n_boxes=20, n_seeds=6, horizon=48, world_seed=9, problem_seed=24)
    R, W, W2 = crgb.Robot(rb), crgb.World(w), crgb.World(w2)
    s1 = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32, seeds=pr.seeds)
    s2 = crgb.ProblemSpec(W2, pr2.q_start, pr2.goal, 48, seeds=pr2.seeds)
    ctx = crgb.Context(0)
    both = crgb.time_discretized_solve(ctx, R, [s1, s2], iters=(10, 10))
    alone = [crgb.time_discretized_solve(ctx, R, s, iters=(10, 10)) for s in (s1, s2)]
    torch.cuda.synchronize()
    for (ob, tb), (oa, ta) in zip(both, alone):
        for k in ("traj", "cost", "cfree", "best"):
            assert torch.equal(getattr(ob, k), getattr(oa, k)), k
        for k in ("first", "stage", "dt", "score", "chosen"):
            assert torch.equal(getattr(tb, k), getattr(ta, k)), k


def test_rank_seeds_matches_oracle():
    """Seed choice of App. "Solver details" (cr_rank_seeds) against the oracle:
    trajectory rule with per-seed time steps and with the params' dt, and the
    IK rule; scores within FP32 rounding, the same chosen index unless the two
    best scores are within that rounding."""
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=8, n_seeds=24, horizon=40, problem_seed=31)
    R, W = crgb.Robot(rb), crgb.World(w)
    rng = np.random.default_rng(32)
    theta = f32(pr.seeds + 0.05 * rng.standard_normal(pr.seeds.shape))
    cfree = (rng.uniform(size=24) < 0.6).astype(np.uint8)
    cfree[:2] = [0, 1]
    dts = f32(rng.uniform(0.02, 0.1, 24))
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 40)
    th = torch.tensor(theta, dtype=torch.float32, device="cuda")
    cf = torch.tensor(cfree, device="cuda")
    cases = [(dict(), torch.tensor(dts, device="cuda"), dict(dt=dts)),
             (dict(dt=0.05), None, dict(dt_all=np.float32(0.05)))]
    for params, dt_dev, ora in cases:
        score, best = crgb.rank_seeds(R, spec, th, cf, params, dt=dt_dev)
        ref, rbest = oracle.rank_seeds(rb, pr.q_start, pr.goal, theta, cfree, **ora, **crgb.RANK_WEIGHTS)
        s = score.cpu().numpy()
        np.testing.assert_allclose(s, ref, rtol=1e-4, atol=1e-6)
        ok = np.where(cfree.astype(bool), ref, np.inf)
        second = np.partition(ok, 1)[1]
        if second - ok[rbest] > 1e-4 * abs(ok[rbest]):
            assert int(best) == rbest
    # IK rule on single states
    q = f32(synth.uniform_config(rng, rb, 50)[:, None, :])
    ispec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 1)
    icf = np.ones(50, dtype=np.uint8)
    score, best = crgb.rank_seeds(R, ispec, torch.tensor(q, dtype=torch.float32, device="cuda"),
                                  torch.tensor(icf, device="cuda"), dict(flags=crgb.IK_MODE))
    ref, rbest = oracle.rank_seeds(rb, pr.q_start, pr.goal, q, icf, ik=True, **crgb.RANK_WEIGHTS)
    np.testing.assert_allclose(score.cpu().numpy(), ref, rtol=1e-4, atol=1e-6)
    assert int(best) == rbest
    # no collision-free seed
    _, best = crgb.rank_seeds(R, spec, th, torch.zeros(24, dtype=torch.uint8, device="cuda"), dict(dt=0.05))
    assert int(best) == -1
