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
    out, dt_opt, dt_f = crgb.time_discretized_solve(ctx, R, spec, iters=(20, 20))
    torch.cuda.synchronize()
    assert 0.0 < dt_opt < 0.25 * 4 and dt_f > 0.0
    b = int(out.best)
    x = out.traj[b].cpu().numpy().astype(np.float64)
    # retimed to dt_f the final trajectory sits at its limits (oracle stencils)
    v, a, j = oracle.stencil(pr.q_start, x, dt_f)
    ratio = max(np.max(np.abs(v) / rb.v_max), np.max(np.abs(a) / rb.a_max), np.max(np.abs(j) / rb.j_max))
    assert ratio == pytest.approx(1.0, rel=1e-4)
    assert np.isfinite(out.cost.cpu().numpy()).all()
