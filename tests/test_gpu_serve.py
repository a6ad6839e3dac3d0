"""Serving: requests of two kinds admitted while others run, state resident on
the device; each result is bit-identical to the same request solved alone."""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_17274_gb300 import crgb, synth

from scenes import f32, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2310_17274_gb300 import build
    build.build_library()
    assert torch.cuda.is_available()
    rb = scene(spheres=synth.SPHERES_60)[0]
    return crgb.Context(0), rb, crgb.Robot(rb)


def _requests(rb, n_mg, n_ik, seed):
    out, keep = [], []
    for k in range(n_mg):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=10 + 7 * k, n_seeds=4, horizon=32,
                         world_seed=seed + k, problem_seed=seed + 50 + k)
        W = crgb.World(w)
        keep.append(W)
        out.append((crgb.MG, crgb.ProblemSpec(W, pr.q_start, pr.goal, 32, seeds=pr.seeds)))
    _, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=20, world_seed=seed + 99)
    W = crgb.World(w)
    keep.append(W)
    for pr in synth.make_ik_problems(rb, w, seed, n_ik, 8, lambda q: oracle.goal_pose_from_fk(rb, q)):
        out.append((crgb.IK, crgb.ProblemSpec(W, f32(pr.q_start), f32(pr.goal), 1, seeds=f32(pr.seeds))))
    return out, keep


IKP = dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE)


def test_served_results_equal_alone(env):
    ctx, rb, R = env
    sv = crgb.Server(ctx, R, mg=(4, 32, 10), ik=(8, 1, 10), ik_params=IKP, chunk=5)
    reqs, keep = _requests(rb, 4, 5, seed=300)
    order = [0, 4, 1, 5, 6, 2, 7, 3, 8]
    tickets = {}
    # staggered arrivals: two requests, a step, two more, ...
    for n, i in enumerate(order):
        tickets[i] = sv.submit(*reqs[i])
        if n % 2 == 1:
            sv.step()
    results = {}
    for _ in range(20):
        for i, t in tickets.items():
            if i not in results:
                r = sv.poll(t)
                if r is not None:
                    results[i] = r
        if len(results) == len(tickets):
            break
        sv.step()
    assert len(results) == len(tickets)
    for i, (kind, spec) in enumerate(reqs):
        p = None if kind == crgb.MG else IKP
        alone = crgb.solve(ctx, R, [spec], p, iters=10, graph=False, persistent=False)[0]
        torch.cuda.synchronize()
        r = results[i]
        np.testing.assert_array_equal(r["traj"], alone.traj.cpu().numpy())
        np.testing.assert_array_equal(r["cost"], alone.cost.cpu().numpy())
        np.testing.assert_array_equal(r["cfree"], alone.cfree.cpu().numpy().astype(bool))
        assert r["best"] == int(alone.best)


def test_admission_waits_for_a_slot(env):
    ctx, rb, R = env
    sv = crgb.Server(ctx, R, mg=(4, 32, 10), ik=(8, 1, 10), ik_params=IKP, chunk=10, max_active=1)
    reqs, keep = _requests(rb, 2, 0, seed=400)
    t0 = sv.submit(*reqs[0])
    t1 = sv.submit(*reqs[1])
    sv.step()                      # admits the first only, runs all its 10 iterations
    assert sv.poll(t0) is not None and sv.poll(t1) is None
    assert sv.stats()["queued"] == 1 and sv.stats()["active"] == 0
    sv.step()
    assert sv.poll(t1) is not None
    assert sv.stats()["active"] == 0


def test_admission_refused_by_memory_reserve(env):
    """A reserve larger than the device keeps every request queued."""
    ctx, rb, R = env
    free, total = torch.cuda.mem_get_info()
    sv = crgb.Server(ctx, R, mg=(4, 32, 10), ik=(8, 1, 10), ik_params=IKP, chunk=10,
                     reserve_bytes=total * 2)
    reqs, keep = _requests(rb, 1, 0, seed=500)
    t = sv.submit(*reqs[0])
    sv.step()
    assert sv.poll(t) is None
    st = sv.stats()
    assert st["queued"] == 1 and st["active"] == 0 and st["pool_bytes"] == 0


def test_submit_rejects_wrong_shape(env):
    ctx, rb, R = env
    sv = crgb.Server(ctx, R, mg=(4, 32, 10), ik=(8, 1, 10), ik_params=IKP, chunk=5)
    reqs, keep = _requests(rb, 1, 0, seed=600)
    kind, spec = reqs[0]
    with pytest.raises(crgb.CrError, match="takes"):
        sv.submit(crgb.IK, spec)
