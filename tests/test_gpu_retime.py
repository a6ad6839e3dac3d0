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


def test_time_discretized_solve():
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=8, n_seeds=8, horizon=32, problem_seed=22)
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32, seeds=pr.seeds)
    ctx = crgb.Context(0)
    out, dt_opt, dt_f, b = crgb.time_discretized_solve(ctx, R, spec, iters=(20, 20))
    torch.cuda.synchronize()
    assert 0.0 < dt_opt < 0.25 * 4 and dt_f > 0.0
    cf = out.cfree.cpu().numpy().astype(bool)
    assert (b >= 0 and cf[b]) if cf.any() else b == max(int(out.best), 0)
    x = out.traj[b].cpu().numpy().astype(np.float64)
    # retimed to dt_f the final trajectory sits at its limits (oracle stencils)
    v, a, j = oracle.stencil(pr.q_start, x, dt_f)
    ratio = max(np.max(np.abs(v) / rb.v_max), np.max(np.abs(a) / rb.a_max), np.max(np.abs(j) / rb.j_max))
    assert ratio == pytest.approx(1.0, rel=1e-4)
    assert np.isfinite(out.cost.cpu().numpy()).all()


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
