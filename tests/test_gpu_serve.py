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


def _requests(rb, n_mg, n_ik, seed, mg_shapes=((4, 32),), ik_seeds=(8,)):
    """n_mg motion-generation requests cycling through mg_shapes (seeds,
    horizon) and n_ik IK requests cycling through ik_seeds."""
    out, keep = [], []
    for k in range(n_mg):
        B, H = mg_shapes[k % len(mg_shapes)]
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=10 + 7 * k, n_seeds=B, horizon=H,
                         world_seed=seed + k, problem_seed=seed + 50 + k)
        W = crgb.World(w)
        keep.append(W)
        out.append((crgb.MG, crgb.ProblemSpec(W, pr.q_start, pr.goal, H, seeds=pr.seeds)))
    _, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=20, world_seed=seed + 99)
    W = crgb.World(w)
    keep.append(W)
    for k in range(n_ik):
        B = ik_seeds[k % len(ik_seeds)]
        pr = synth.make_ik_problems(rb, w, seed + k, 1, B, lambda q: oracle.goal_pose_from_fk(rb, q))[0]
        out.append((crgb.IK, crgb.ProblemSpec(W, f32(pr.q_start), f32(pr.goal), 1, seeds=f32(pr.seeds))))
    return out, keep


IKP = dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE)


def _drain(sv, tickets, limit_s=60.0):
    import time
    t0 = time.time()
    results = {}
    while len(results) < len(tickets):
        sv.step()
        for i, t in tickets.items():
            if i not in results:
                r = sv.poll(t)
                if r is not None:
                    results[i] = r
        assert time.time() - t0 < limit_s, "server did not finish"
    return results


def _alone(ctx, R, kind, spec, iters=10):
    p = None if kind == crgb.MG else IKP
    o = crgb.solve(ctx, R, [spec], p, iters=iters, graph=False, persistent=False)[0]
    torch.cuda.synchronize()
    return o


def _same(r, alone):
    np.testing.assert_array_equal(r["traj"], alone.traj.cpu().numpy())
    np.testing.assert_array_equal(r["cost"], alone.cost.cpu().numpy())
    np.testing.assert_array_equal(r["cfree"], alone.cfree.cpu().numpy().astype(bool))
    assert r["best"] == int(alone.best)
    assert r["status"] == int(alone.status)


def test_served_results_equal_alone(env):
    """Requests of different sizes within each kind (motion generation 4 x 32,
    6 x 24 and 3 x 48; IK 8 and 5 seeds), arriving while others run: each
    result equals the request solved alone, bit for bit."""
    ctx, rb, R = env
    sv = crgb.Server(ctx, R, mg_iters=10, ik_iters=10, ik_params=IKP, chunk=5)
    reqs, keep = _requests(rb, 5, 5, seed=300, mg_shapes=((4, 32), (6, 24), (3, 48)), ik_seeds=(8, 5))
    order = [0, 5, 1, 6, 7, 2, 8, 3, 9, 4]
    tickets = {}
    # staggered arrivals: two requests, a step, two more, ...
    for n, i in enumerate(order):
        tickets[i] = sv.submit(*reqs[i])
        if n % 2 == 1:
            sv.step()
    results = _drain(sv, tickets)
    for i, (kind, spec) in enumerate(reqs):
        _same(results[i], _alone(ctx, R, kind, spec))


def test_admission_waits_for_a_slot(env):
    ctx, rb, R = env
    sv = crgb.Server(ctx, R, mg_iters=10, ik_iters=10, ik_params=IKP, chunk=10, max_active=1)
    reqs, keep = _requests(rb, 2, 0, seed=400)
    t0 = sv.submit(*reqs[0])
    t1 = sv.submit(*reqs[1])
    sv.step()                      # admits the first only and starts its round
    st = sv.stats()
    assert st["queued"] == 1 and st["active"] == 1
    r0 = sv.wait(t0)
    assert r0 is not None
    r1 = sv.wait(t1)
    assert r1 is not None and sv.stats()["active"] == 0
    _same(r1, _alone(ctx, R, *reqs[1]))


def test_admission_refused_by_memory_reserve_times_out(env):
    """A reserve larger than the device keeps every request queued; waiting
    for it ends with CR_ETIMEOUT."""
    ctx, rb, R = env
    free, total = torch.cuda.mem_get_info()
    sv = crgb.Server(ctx, R, mg_iters=10, ik_iters=10, ik_params=IKP, chunk=10, reserve_bytes=total * 2)
    reqs, keep = _requests(rb, 1, 0, seed=500)
    t = sv.submit(*reqs[0])
    with pytest.raises(crgb.CrError) as e:
        sv.wait(t, timeout_ms=50)
    assert e.value.status == crgb.ETIMEOUT
    assert sv.poll(t) is None
    st = sv.stats()
    assert st["queued"] == 1 and st["active"] == 0 and st["pool_bytes"] == 0


def test_submit_limits(env):
    """A full queue refuses a request with CR_EBUSY; an IK request must have
    horizon 1."""
    ctx, rb, R = env
    sv = crgb.Server(ctx, R, mg_iters=10, ik_iters=10, ik_params=IKP, chunk=5, max_queued=2)
    reqs, keep = _requests(rb, 3, 0, seed=600)
    sv.submit(*reqs[0])
    sv.submit(*reqs[1])
    with pytest.raises(crgb.CrError) as e:
        sv.submit(*reqs[2])
    assert e.value.status == crgb.EBUSY
    with pytest.raises(crgb.CrError, match="horizon 1"):
        sv.submit(crgb.IK, reqs[2][1])


def test_snapshot_restore_bit_identical(env):
    """A request's device optimiser state copied out mid-solve (after the
    first of four rounds) and restored into a fresh server finishes with
    exactly the bits of the uninterrupted request and of the request solved
    alone; a request snapshot while still queued restores as a new one."""
    ctx, rb, R = env
    reqs, keep = _requests(rb, 2, 1, seed=700)
    a = crgb.Server(ctx, R, mg_iters=20, ik_iters=20, ik_params=IKP, chunk=5)
    b = crgb.Server(ctx, R, mg_iters=20, ik_iters=20, ik_params=IKP, chunk=5)
    ta = {i: a.submit(*reqs[i]) for i in (0, 2)}
    a.step()                              # admitted, first round (5 iterations) running
    blobs = {i: a.snapshot(ta[i]) for i in (0, 2)}   # waits for that round
    queued = a.submit(*reqs[1])
    blob_q = a.snapshot(queued)                      # still queued: inputs only
    assert len(blob_q) < len(blobs[0])
    worlds = {0: reqs[0][1].world, 1: reqs[1][1].world, 2: reqs[2][1].world}
    tb = {i: b.restore(blobs[i], worlds[i]) for i in (0, 2)}
    tb[1] = b.restore(blob_q, worlds[1])
    ta[1] = queued
    ra = _drain(a, ta)
    rb_ = _drain(b, tb)
    for i in (0, 1, 2):
        for k in ("traj", "cost", "cfree", "best", "status"):
            np.testing.assert_array_equal(ra[i][k], rb_[i][k])
        _same(rb_[i], _alone(ctx, R, *reqs[i], iters=20))
    # a snapshot does not fit a server with other parameters
    c = crgb.Server(ctx, R, mg_iters=20, ik_iters=20, ik_params=IKP, chunk=5, mg_params=dict(eta=0.03))
    with pytest.raises(crgb.CrError, match="parameters"):
        c.restore(blobs[0], worlds[0])


def test_served_status_word(env):
    """A request with a NaN in a seed finishes with CR_ENAN; the request
    served beside it is unaffected."""
    ctx, rb, R = env
    reqs, keep = _requests(rb, 2, 0, seed=800)
    kind, spec = reqs[1]
    bad_seeds = spec.seeds.copy()
    bad_seeds[0, 3, 2] = np.nan
    bad = crgb.ProblemSpec(spec.world, spec.q_start, spec.goal, spec.horizon, seeds=bad_seeds)
    sv = crgb.Server(ctx, R, mg_iters=10, ik_iters=10, ik_params=IKP, chunk=5)
    t = {0: sv.submit(*reqs[0]), 1: sv.submit(kind, bad)}
    res = _drain(sv, t)
    assert res[1]["status"] == crgb.ENAN and res[0]["status"] == crgb.OK
    _same(res[0], _alone(ctx, R, *reqs[0]))
