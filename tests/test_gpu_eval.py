"""GPU parity of forward kinematics and of the fused cost-and-gradient kernel
against the FP64 oracle, through the C ABI.

Tolerances (FP32 GPU vs FP64 oracle on the same float32-rounded inputs):
  sphere centres |d| <= 1e-5 m; costs |d| <= 1e-4 max(|ref|, 1e-2) per term and
  total; gradient per trajectory ||d|| <= 1e-3 ||ref|| + 1e-6; collision-free
  flags bit-exact.

Near-threshold states.  FP32 rounding can flip a discrete decision (a sweep
activation or stop test, a face or pair argmax, the zero of Eq. 9's max) that
the oracle takes within 1e-5 m of its threshold.  The oracle reports, per
state, the margin of the decisions that set that state's world and self cost
and gradient, and its smallest clearance.  A state whose margin is below
1e-5 m is left out state by state: its world and self costs are taken out of
both sides' totals (the kernel writes the same per-state costs), and the
gradient rows it reaches (t - 1, t, t + 1, through the speed metric) are not
compared.  Everything else of the trajectory is compared element-wise, and
every test asserts how many states it compared.  The collision-free flag is
compared whenever the clear states decide it.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2310_17274_gb300 import crgb, synth

from scenes import f32, line_search_batch, scene

pytestmark = pytest.mark.gpu

NEAR = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2310_17274_gb300 import build
    build.build_library()
    oracle.build()
    assert torch.cuda.is_available()


def _gpu_eval(rb, w, pr, theta, params=None, goal_q=None):
    R = crgb.Robot(rb)
    W = crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, theta.shape[1], goal_q=goal_q)
    out = crgb.evaluate(R, spec, torch.tensor(theta, dtype=torch.float32, device="cuda"), params,
                        want_states=True)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def _ref_eval(rb, w, pr, theta, params=None, goal_q=None):
    return oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, params, goal_q=goal_q, states=True)


def _close(g, r):
    return abs(g - r) <= 1e-4 * max(abs(r), 1e-2)


def compare(gpu, ref, min_states=0.5, label=""):
    """The parity bar, state by state (module docstring).  Returns (states
    compared, states); asserts that at least `min_states` of the states were
    compared."""
    B, H = ref["state_margin"].shape
    near = ref["state_margin"] < NEAR
    n_cmp = 0
    n_flag = 0
    for b in range(B):
        nb = near[b]
        keep = ~nb
        n_cmp += int(keep.sum())
        gst, rst = gpu["state_terms"][b].astype(np.float64), ref["state_terms"][b]
        # the kernel's per-state costs add up to its own terms
        for k in (0, 1):
            assert abs(gst[:, k].sum() - gpu["terms"][b, k]) <= 1e-5 * max(abs(gpu["terms"][b, k]), 1e-1), \
                (label, b, k, gst[:, k].sum(), gpu["terms"][b, k])
        # world and self cost over the clear states
        for k in (0, 1):
            g, r = gst[keep, k].sum(), rst[keep, k].sum()
            assert _close(g, r), (label, b, "term", k, g, r)
        # the terms without discrete decisions
        for k in (2, 3, 4):
            assert _close(gpu["terms"][b, k], ref["terms"][b, k]), \
                (label, b, "term", k, gpu["terms"][b, k], ref["terms"][b, k])
        # total less the near states' world and self costs, each side its own
        g = float(gpu["cost"][b]) - gst[nb].sum()
        r = float(ref["cost"][b]) - rst[nb].sum()
        assert _close(g, r), (label, b, "cost", g, r)
        # gradient rows out of reach of every near decision
        if gpu.get("grad") is not None and ref.get("grad") is not None:
            reach = nb.copy()
            reach[1:] |= nb[:-1]
            reach[:-1] |= nb[1:]
            rows = ~reach
            if rows.any():
                gg, rg = gpu["grad"][b][rows], ref["grad"][b][rows]
                err = np.linalg.norm(gg - rg)
                assert err <= 1e-3 * np.linalg.norm(rg) + 1e-6, (label, b, err, np.linalg.norm(rg))
        # the flag, when the clear states decide it
        cl = ref["state_clear"][b]
        sure = np.abs(cl) >= NEAR
        if (cl[sure] < 0).any():
            expect = False
        elif sure.all():
            expect = bool(ref["cfree"][b])
        else:
            continue
        n_flag += 1
        assert bool(gpu["cfree"][b]) == expect, (label, b)
    assert n_cmp >= min_states * B * H, f"{label}: compared {n_cmp} of {B * H} states"
    return n_cmp, B * H


# ---------------------------------------------------------------------------
# forward kinematics
# ---------------------------------------------------------------------------

def test_fk_parity():
    rb, _, _ = scene(spheres=synth.SPHERES_60)
    rng = np.random.default_rng(0)
    q = f32(synth.uniform_config(rng, rb, 300))
    R = crgb.Robot(rb)
    sp, ee, lt = crgb.fk(R, torch.tensor(q, dtype=torch.float32, device="cuda"), link_tf=True)
    sp, ee, lt = sp.cpu().numpy(), ee.cpu().numpy(), lt.cpu().numpy()
    for n in range(len(q)):
        lt_r, sp_r, ee_r = oracle.fk(rb, q[n])
        assert np.abs(sp[n, :, :3] - sp_r[:, :3]).max() <= 1e-5
        assert np.array_equal(sp[n, :, 3], sp_r[:, 3].astype(np.float32))
        assert np.abs(ee[n] - ee_r).max() <= 1e-5
        assert np.abs(lt[n] - lt_r).max() <= 1e-5


def test_fk_empty_and_single():
    rb, _, _ = scene()
    R = crgb.Robot(rb)
    sp, ee, _ = crgb.fk(R, torch.zeros((0, rb.dof), device="cuda"))
    assert sp.shape[0] == 0
    sp, ee, _ = crgb.fk(R, torch.zeros((1, rb.dof), device="cuda"))
    _, sp_r, ee_r = oracle.fk(rb, np.zeros(rb.dof))
    assert np.abs(sp.cpu().numpy()[0, :, :3] - sp_r[:, :3]).max() <= 1e-6


# ---------------------------------------------------------------------------
# fused evaluation
# ---------------------------------------------------------------------------

def test_eval_parity_tiny():
    """Tiny workload: 7-DOF, 42 spheres, 8 boxes, 4 seeds x 4 step sizes x 32 steps."""
    rb, w, pr = scene()
    theta = line_search_batch(pr, np.random.default_rng(1))
    gpu = _gpu_eval(rb, w, pr, theta)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, states=True)
    assert np.any(ref["terms"][:, 0] > 0), "world term inactive: scene too easy"
    compare(gpu, ref, min_states=0.9, label="tiny")


@pytest.mark.parametrize("flags", [
    crgb.SPEED | crgb.SELF,                      # sweep off
    crgb.SWEPT | crgb.SELF,                      # speed off
    crgb.SWEPT | crgb.SPEED,                     # self off
    crgb.SWEPT | crgb.SPEED | crgb.SELF | crgb.VEL_COST,
])
def test_eval_parity_flags(flags):
    rb, w, pr = scene(n_boxes=12, world_seed=3, problem_seed=4)
    theta = line_search_batch(pr, np.random.default_rng(2))
    p = dict(flags=flags | crgb.WOLFE)
    gpu = _gpu_eval(rb, w, pr, theta, p)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, p, states=True)
    compare(gpu, ref, label=f"flags={flags}")


@pytest.mark.parametrize("horizon,ik", [(32, False), (1, True)])
def test_eval_parity_cspace_goal(horizon, ik):
    """Eq. 15 joint-space goal cost at the last state (trajectories and IK)."""
    rb, w, pr = scene(n_boxes=6, n_seeds=4, horizon=horizon, world_seed=5, problem_seed=6)
    rng = np.random.default_rng(7)
    # a goal pose away from every last state: near a reached pose the Eq. 14
    # cost is steep in the end-effector position and FP32 kinematics error
    # shows; Eq. 15 is what this test is about
    pr.goal = f32(oracle.goal_pose_from_fk(rb, synth.uniform_config(rng, rb)))
    goal_q = f32(pr.seeds[0, -1] + rng.normal(0, 0.3, size=rb.dof))
    theta = line_search_batch(pr, rng, scale=0.1)
    flags = (crgb.IK_MODE | crgb.SELF if ik else crgb.SWEPT | crgb.SPEED | crgb.SELF) | crgb.WOLFE
    p = dict(flags=flags | crgb.CSPACE_GOAL)
    gpu = _gpu_eval(rb, w, pr, theta, p, goal_q=goal_q)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, p, goal_q=goal_q, states=True)
    compare(gpu, ref, min_states=0.8, label=f"cspace H={horizon}")
    # the flag without a goal configuration, and a goal configuration without the flag, add nothing
    plain = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, dict(flags=flags), states=True)
    g1 = _gpu_eval(rb, w, pr, theta, p)
    g2 = _gpu_eval(rb, w, pr, theta, dict(flags=flags), goal_q=goal_q)
    compare(g1, plain, label="flag only")
    compare(g2, plain, label="goal only")


def test_eval_parity_trajopt_shape():
    """Trajectory-optimisation shape: 60 spheres, 32 boxes, H = 48 (8 trajectories)."""
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=32, n_seeds=4, horizon=48, world_seed=2,
                      problem_seed=11)
    theta = line_search_batch(pr, np.random.default_rng(3), alphas=(0.1, 0.5))
    gpu = _gpu_eval(rb, w, pr, theta, dict(alpha=list(synth.ALPHA_8)))
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, states=True)
    compare(gpu, ref, min_states=0.8, label="trajopt")


def test_eval_parity_ik():
    """IK shape: H = 1, IK mode, 60 spheres, 40 boxes, a ragged batch of 50."""
    rb, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=40, world_seed=3)
    rng = np.random.default_rng(5)
    qg = synth.uniform_config(rng, rb)
    goal = f32(oracle.goal_pose_from_fk(rb, qg))
    theta = f32(synth.uniform_config(rng, rb, 50)[:, None, :])
    pr = synth.Problem(world=w, q_start=f32(synth.uniform_config(rng, rb)), goal=goal, seeds=theta)
    p = dict(flags=crgb.IK_MODE | crgb.SELF)
    gpu = _gpu_eval(rb, w, pr, theta, p)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, p, states=True)
    compare(gpu, ref, min_states=0.8, label="ik")
    assert gpu["cfree"].any() and not gpu["cfree"].all()


@pytest.mark.parametrize("spheres, horizon", [(synth.SPHERES_60, 3), ((12, 12, 12, 12, 12, 12, 12), 1)])
def test_eval_parity_ik_paths(spheres, horizon):
    """IK mode on the per-trajectory kernel: several independent states per
    trajectory (costs summed, pose goal at the last one), and a robot of 84
    spheres (more than the pair table covers: every listed pair of a close
    link pair is visited); 70 boxes (two chunks of the link box masks)."""
    rb, w, _ = scene(spheres=spheres, n_boxes=70, world_seed=11)
    rng = np.random.default_rng(12)
    goal = f32(oracle.goal_pose_from_fk(rb, synth.uniform_config(rng, rb)))
    theta = f32(synth.uniform_config(rng, rb, 37 * horizon).reshape(37, horizon, rb.dof))
    pr = synth.Problem(world=w, q_start=f32(synth.uniform_config(rng, rb)), goal=goal, seeds=theta)
    p = dict(flags=crgb.IK_MODE | crgb.SELF)
    gpu = _gpu_eval(rb, w, pr, theta, p)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta, p, states=True)
    compare(gpu, ref, min_states=0.7, label=f"ik paths {len(spheres)} {horizon}")


def test_eval_ik_small_and_large_launches_agree():
    """IK mode: a small launch runs several threads per trajectory, a large
    one a thread each; the same trajectories give the same bits either way."""
    rb, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=40, world_seed=21)
    R, W = crgb.Robot(rb), crgb.World(w)
    rng = np.random.default_rng(22)
    goal = f32(oracle.goal_pose_from_fk(rb, synth.uniform_config(rng, rb)))
    q = torch.tensor(synth.uniform_config(rng, rb, 20000)[:, None, :], dtype=torch.float32, device="cuda")
    spec = crgb.ProblemSpec(W, f32(synth.uniform_config(rng, rb)), goal, 1)
    p = dict(flags=crgb.IK_MODE | crgb.SELF)
    small = crgb.evaluate(R, spec, q[:100].contiguous(), p)
    large = crgb.evaluate(R, spec, q, p)
    # cost-only launches (steering, particles) take the same arithmetic
    small_nog = crgb.evaluate(R, spec, q[:100].contiguous(), p, want_grad=False)
    large_nog = crgb.evaluate(R, spec, q, p, want_grad=False)
    torch.cuda.synchronize()
    for k in ("cost", "grad", "cfree", "terms"):
        assert torch.equal(small[k], large[k][:100]), k
    for k in ("cost", "cfree", "terms"):
        assert torch.equal(small[k], small_nog[k]) and torch.equal(large[k], large_nog[k]), k
    assert 0 < int(large["cfree"].sum()) < 20000


def test_eval_ik_twelve_joints():
    """IK mode on a 12-joint chain (more links than threads per trajectory in
    the split form, so a thread owns two links): parity with the oracle in a
    small launch, and the same bits in a large one."""
    from scenes import as_f32_robot, as_f32_world
    rb = as_f32_robot(synth.make_robot((5,) * 12, seed=3, axes=(2, 1) * 6))
    rng = np.random.default_rng(23)
    w = as_f32_world(synth.make_world(30, 24))
    goal = f32(oracle.goal_pose_from_fk(rb, synth.uniform_config(rng, rb)))
    q = f32(synth.uniform_config(rng, rb, 20000)[:, None, :])
    pr = synth.Problem(world=w, q_start=f32(synth.uniform_config(rng, rb)), goal=goal, seeds=q[:60])
    p = dict(flags=crgb.IK_MODE | crgb.SELF)
    gpu = _gpu_eval(rb, w, pr, q[:60], p)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, q[:60], p, states=True)
    compare(gpu, ref, min_states=0.7, label="ik 12 joints")
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, goal, 1)
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    small = crgb.evaluate(R, spec, qd[:60].contiguous(), p)
    large = crgb.evaluate(R, spec, qd, p)
    torch.cuda.synchronize()
    for k in ("cost", "grad", "cfree", "terms"):
        assert torch.equal(small[k], large[k][:60]), k


def test_eval_parity_ik_self_contact():
    """IK mode, no boxes: configurations folded onto themselves so that many
    states have penetrating sphere pairs (the self term's argmax and its
    gradient, and the collision-free flag from self contact alone)."""
    rb, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=0)
    rng = np.random.default_rng(13)
    lo, hi = np.asarray(rb.q_lo), np.asarray(rb.q_hi)
    # joints pushed towards their limits fold the chain
    u = rng.uniform(0.0, 1.0, (300, rb.dof)) ** 0.25 * np.where(rng.uniform(size=(300, rb.dof)) < 0.5, -1, 1)
    q = f32(0.5 * (lo + hi) + 0.5 * (hi - lo) * u)[:, None, :]
    goal = f32(oracle.goal_pose_from_fk(rb, synth.uniform_config(rng, rb)))
    pr = synth.Problem(world=w, q_start=f32(synth.uniform_config(rng, rb)), goal=goal, seeds=q)
    p = dict(flags=crgb.IK_MODE | crgb.SELF)
    gpu = _gpu_eval(rb, w, pr, q, p)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, q, p, states=True)
    compare(gpu, ref, min_states=0.7, label="ik self contact")
    hit = ref["terms"][:, 1] > 0
    assert hit.sum() >= 20 and (~hit).sum() >= 20, hit.sum()


def test_eval_ik_without_self_check():
    """IK without collision checking: the no-self-check flag drops self contact
    from the collision-free flag (parity with the oracle on folded
    configurations, costs unchanged) and is refused outside IK mode or with
    the self term on."""
    rb, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=0)
    rng = np.random.default_rng(14)
    lo, hi = np.asarray(rb.q_lo), np.asarray(rb.q_hi)
    u = rng.uniform(0.0, 1.0, (200, rb.dof)) ** 0.25 * np.where(rng.uniform(size=(200, rb.dof)) < 0.5, -1, 1)
    q = f32(0.5 * (lo + hi) + 0.5 * (hi - lo) * u)[:, None, :]
    goal = f32(oracle.goal_pose_from_fk(rb, synth.uniform_config(rng, rb)))
    pr = synth.Problem(world=w, q_start=f32(synth.uniform_config(rng, rb)), goal=goal, seeds=q)
    p = dict(flags=crgb.IK_MODE | crgb.NO_SELF_CHECK)
    gpu = _gpu_eval(rb, w, pr, q, p)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, q, p, states=True)
    compare(gpu, ref, label="ik no self check")
    assert gpu["cfree"].all()
    plain = _gpu_eval(rb, w, pr, q, dict(flags=crgb.IK_MODE))
    assert not plain["cfree"].all()
    np.testing.assert_array_equal(plain["cost"], gpu["cost"])
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, goal, 1)
    th = torch.tensor(q, dtype=torch.float32, device="cuda")
    for bad in (crgb.NO_SELF_CHECK, crgb.IK_MODE | crgb.SELF | crgb.NO_SELF_CHECK):
        with pytest.raises(crgb.CrError):
            crgb.evaluate(R, spec, th, dict(flags=bad))


@pytest.mark.parametrize("K,H,spheres", [(100, 64, synth.SPHERES_60), (200, 64, synth.SPHERES_60),
                                         (200, 96, synth.SPHERES_60), (100, 128, synth.SPHERES_42),
                                         (200, 128, synth.SPHERES_42)])
def test_eval_many_boxes_long_horizons(K, H, spheres):
    """More boxes than one shared-memory chunk (100 and 200 > 64: two and four
    chunks of the link box masks) at long horizons: 64 and 96 on the
    trajectory-optimisation robot (60 spheres), 128 (the largest) on the
    42-sphere robot (a whole trajectory of 128 states with 60 spheres needs
    more shared memory than a CTA has, which the library refuses):
    state-by-state parity, at least 80 % of the states compared, the world
    term active."""
    rb, w, pr = scene(spheres=spheres, n_boxes=K, n_seeds=2, horizon=H, world_seed=8 + K,
                      problem_seed=3 + H)
    theta = line_search_batch(pr, np.random.default_rng(K + H), alphas=(0.3, 1.0), scale=0.1)
    gpu = _gpu_eval(rb, w, pr, theta)
    ref = _ref_eval(rb, w, pr, theta)
    active = ref["state_terms"][:, :, 0] > 0
    assert active.sum() >= 10, active.sum()
    compare(gpu, ref, min_states=0.8, label=f"K={K},H={H},M={len(rb.spheres)}")


def test_eval_refuses_a_tile_beyond_shared_memory():
    """60 spheres x 128 states in one trajectory tile exceed the CTA's shared
    memory: a clear CR_EINVAL, no launch."""
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=4, n_seeds=1, horizon=128)
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 128)
    with pytest.raises(crgb.CrError, match="shared memory"):
        crgb.evaluate(R, spec, torch.tensor(pr.seeds, dtype=torch.float32, device="cuda"))


def test_eval_edge_cases():
    rb, w, pr = scene(n_seeds=3, horizon=5)
    # no boxes
    w0 = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    gpu = _gpu_eval(rb, w0, pr, pr.seeds)
    ref = oracle.evaluate(rb, w0, pr.q_start, pr.goal, pr.seeds, states=True)
    compare(gpu, ref, min_states=0.9, label="K=0")
    assert np.all(gpu["terms"][:, 0] == 0)
    # H = 1 outside IK mode (stencil over one state) and H = 2
    for H in (1, 2):
        th = pr.seeds[:, :H].copy()
        gpu = _gpu_eval(rb, w, pr, th)
        ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, th, states=True)
        compare(gpu, ref, min_states=0.6, label=f"H={H}")
    # disabled spheres (negative radius)
    rb2 = synth.Robot(**{**rb.__dict__, "spheres": rb.spheres.copy()})
    rb2.spheres[::3, 3] = -1.0
    gpu = _gpu_eval(rb2, w, pr, pr.seeds)
    ref = oracle.evaluate(rb2, w, pr.q_start, pr.goal, pr.seeds, states=True)
    compare(gpu, ref, min_states=0.8, label="disabled spheres")
    # empty batch is a no-op
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 5)
    out = crgb.evaluate(R, spec, torch.zeros((0, 5, rb.dof), device="cuda"))
    assert out["cost"].numel() == 0


def test_eval_rejects_bad_sizes():
    rb, w, pr = scene()
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 129)
    with pytest.raises(crgb.CrError, match="horizon"):
        crgb.evaluate(R, spec, torch.zeros((1, 129, rb.dof), device="cuda"))
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 4)
    with pytest.raises(crgb.CrError, match="history"):
        crgb.evaluate(R, spec, torch.zeros((1, 4, rb.dof), device="cuda"), dict(history=0))


def test_eval_deterministic_and_batch_independent():
    """Same inputs give bit-identical outputs, and a trajectory's result does
    not depend on what else is in the batch."""
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=32, n_seeds=8, horizon=48, world_seed=2)
    theta = line_search_batch(pr, np.random.default_rng(7))
    a = _gpu_eval(rb, w, pr, theta)
    b = _gpu_eval(rb, w, pr, theta)
    for k in ("cost", "grad", "cfree", "terms"):
        assert np.array_equal(a[k], b[k]), k
    sub = _gpu_eval(rb, w, pr, theta[5:9])
    for k in ("cost", "grad", "cfree", "terms"):
        assert np.array_equal(a[k][5:9], sub[k]), k


def test_eval_full_size_sampled():
    """Bench configuration (60 spheres, 32 boxes, 32 seeds x 8 step sizes x 48
    steps in one launch): sampled trajectories against the oracle, and
    cost = sum of terms everywhere."""
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=32, n_seeds=32, horizon=48,
                      world_seed=2, problem_seed=2)
    theta = line_search_batch(pr, np.random.default_rng(9), alphas=synth.ALPHA_8)
    assert theta.shape == (256, 48, 7)
    gpu = _gpu_eval(rb, w, pr, theta)
    np.testing.assert_allclose(gpu["cost"], gpu["terms"].sum(1), rtol=1e-5)
    idx = np.random.default_rng(0).choice(256, 10, replace=False)
    ref = oracle.evaluate(rb, w, pr.q_start, pr.goal, theta[idx], states=True)
    compare({k: v[idx] for k, v in gpu.items()}, ref, min_states=0.8, label="full-size sample")


def test_autograd_matches_oracle_finite_differences():
    """Gradient through torch.autograd.Function equals central finite
    differences (h = 1e-4, FP64) of the oracle's cost (sweep off: its
    gradient is a surrogate by design)."""
    from paper_2310_17274_gb300.autograd import trajectory_cost
    rb, w, pr = scene(n_boxes=10, n_seeds=2, horizon=8, world_seed=5, problem_seed=5)
    p = dict(flags=crgb.SPEED | crgb.SELF | crgb.WOLFE)
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 8)
    th = torch.tensor(pr.seeds, dtype=torch.float32, device="cuda", requires_grad=True)
    cost = trajectory_cost(th, R, spec, crgb.make_params(p))
    (cost * torch.tensor([1.0, 2.0], device="cuda")).sum().backward()
    g = th.grad.cpu().numpy()
    h = 1e-4
    num = np.zeros_like(pr.seeds)
    for b in range(2):
        for t in range(8):
            for j in range(rb.dof):
                tp, tm = pr.seeds[b:b + 1].copy(), pr.seeds[b:b + 1].copy()
                tp[0, t, j] += h
                tm[0, t, j] -= h
                cp = oracle.evaluate(rb, w, pr.q_start, pr.goal, tp, p, want_grad=False)["cost"][0]
                cm = oracle.evaluate(rb, w, pr.q_start, pr.goal, tm, p, want_grad=False)["cost"][0]
                num[b, t, j] = (cp - cm) / (2 * h) * (1.0 + b)
    for b in range(2):
        err = np.linalg.norm(g[b] - num[b])
        assert err <= 1e-3 * np.linalg.norm(num[b]) + 1e-6, (b, err, np.linalg.norm(num[b]))
