"""Particle-based optimisation (Sec. 4.2, Eq. 12-13) through cr_particle_step
against the oracle: samples, their costs, the exponential-utility weights and
the mean / covariance updates, one iteration at a time on the same inputs."""
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


def _dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def _check_iteration(rb, w, pr, R, spec, mu, sigma, eps, beta, k_mu, k_s, params=None):
    """One GPU iteration from (mu, sigma) vs the oracle from the same FP32 values."""
    B, n_p = eps.shape[:2]
    H, D = mu.shape[1:]
    n = H * D
    mu_d, sg_d = _dev(mu), _dev(sigma)
    parts, cost = crgb.particle_step(R, spec, mu_d, sg_d, _dev(eps), params=params, beta=beta,
                                     k_mu=k_mu, k_sigma=k_s)
    torch.cuda.synchronize()
    parts = parts.cpu().numpy().astype(np.float64)
    cost = cost.cpu().numpy().astype(np.float64)
    for b in range(B):
        ref_p = oracle.particle_sample(mu[b].ravel(), sigma[b].ravel(), eps[b].reshape(n_p, n))
        np.testing.assert_allclose(parts[b].reshape(n_p, n), ref_p, rtol=1e-6, atol=1e-6)
        # costs of the samples the GPU drew
        ev = oracle.evaluate(rb, w, pr.q_start, pr.goal, parts[b], params)
        ok = ev["margin"] >= 1e-5
        assert np.all(np.abs(cost[b] - ev["cost"])[ok] <= 1e-4 * np.maximum(np.abs(ev["cost"][ok]), 1e-2))
        # the update from the GPU's own costs and samples
        m2, s2, _ = oracle.particle_update(cost[b], parts[b].reshape(n_p, n), mu[b].ravel(),
                                           sigma[b].ravel(), beta, k_mu, k_s)
        scale = np.abs(parts[b]).max() + 1.0
        np.testing.assert_allclose(mu_d[b].cpu().numpy().ravel(), m2, atol=2e-5 * scale)
        np.testing.assert_allclose(sg_d[b].cpu().numpy().ravel(), s2, atol=2e-5 * scale ** 2)
    return mu_d.cpu().numpy().astype(np.float64), sg_d.cpu().numpy().astype(np.float64)


def test_particle_iterations_match_oracle():
    rb, w, pr = scene(n_seeds=3, horizon=32, problem_seed=11)
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32)
    rng = np.random.default_rng(5)
    mu = pr.seeds.copy()
    sigma = f32(np.full_like(mu, 0.01))
    for it, (beta, k_mu, k_s) in enumerate([(50.0, 0.9, 0.9), (5.0, 0.5, 0.7)]):
        eps = f32(rng.standard_normal((3, 8) + mu.shape[1:]))
        mu, sigma = _check_iteration(rb, w, pr, R, spec, mu, sigma, eps, beta, k_mu, k_s)


def test_particle_ik_shape_and_single_particle():
    rb, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=12, n_seeds=5, horizon=1, problem_seed=4)
    R, W = crgb.Robot(rb), crgb.World(w)
    p = dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 1)
    rng = np.random.default_rng(6)
    mu = f32(synth.uniform_config(rng, rb, 5)[:, None, :])
    sigma = f32(np.full_like(mu, 0.04))
    eps = f32(rng.standard_normal((5, 16, 1, rb.dof)))
    _check_iteration(rb, w, pr, R, spec, mu, sigma, eps, 10.0, 1.0, 1.0, params=p)
    # one particle, rates 1: the mean becomes the particle, sigma its squared step
    eps1 = f32(rng.standard_normal((5, 1, 1, rb.dof)))
    mu_d, sg_d = _dev(mu), _dev(sigma)
    parts, _ = crgb.particle_step(R, spec, mu_d, sg_d, _dev(eps1), params=p, beta=1.0, k_mu=1.0,
                                  k_sigma=1.0)
    torch.cuda.synchronize()
    assert torch.allclose(mu_d, parts[:, 0], atol=1e-6)
    assert torch.allclose(sg_d, (parts[:, 0] - _dev(mu)) ** 2, atol=1e-6)


def test_particle_step_is_deterministic_and_seed_independent():
    rb, w, pr = scene(n_seeds=4, horizon=32, problem_seed=13)
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32)
    rng = np.random.default_rng(8)
    eps = f32(rng.standard_normal((4, 6) + pr.seeds.shape[1:]))
    outs = []
    for _ in range(2):
        mu_d, sg_d = _dev(pr.seeds), _dev(np.full_like(pr.seeds, 0.02))
        crgb.particle_step(R, spec, mu_d, sg_d, _dev(eps), beta=20.0)
        torch.cuda.synchronize()
        outs.append((mu_d.clone(), sg_d.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    # seed 2 alone gives what it gave in the batch
    mu_d, sg_d = _dev(pr.seeds[2:3]), _dev(np.full_like(pr.seeds[2:3], 0.02))
    crgb.particle_step(R, spec, mu_d, sg_d, _dev(eps[2:3]), beta=20.0)
    torch.cuda.synchronize()
    assert torch.equal(mu_d[0], outs[0][0][2]) and torch.equal(sg_d[0], outs[0][1][2])


def test_particle_step_rejects_bad_arguments():
    rb, w, pr = scene(n_seeds=1, horizon=32)
    R, W = crgb.Robot(rb), crgb.World(w)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, 32)
    mu = _dev(pr.seeds)
    eps = _dev(np.zeros((1, 2) + pr.seeds.shape[1:]))
    for kw in (dict(beta=0.0), dict(beta=1.0, k_mu=1.5), dict(beta=1.0, k_sigma=-0.1)):
        with pytest.raises(crgb.CrError):
            crgb.particle_step(R, spec, mu, _dev(np.ones_like(pr.seeds)), eps, **kw)


@pytest.mark.parametrize("ik", [False, True])
def test_particles_in_solve_equal_particle_steps(ik):
    """cr_solve_particles: particle iterations over every seed of a batch of
    uneven problems, then L-BFGS, equal bit for bit to cr_particle_step on
    each problem followed by cr_solve from the resulting means (trajectory
    problems of horizons 32 and 20; IK problems of 32 and 12 seeds)."""
    rb = scene(spheres=synth.SPHERES_60)[0]
    R = crgb.Robot(rb)
    ctx = crgb.Context(0)
    shapes = [(12, 32, 1), (20, 12, 1)] if ik else [(10, 4, 32), (25, 3, 20)]
    specs, keep, probs = [], [], []
    for k, (K, B, H) in enumerate(shapes):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=K, n_seeds=B, horizon=max(H, 2), world_seed=70 + k,
                         problem_seed=80 + k)
        seeds = pr.seeds[:, :H].copy() if H > 1 else f32(synth.uniform_config(np.random.default_rng(k), rb, B))[:, None]
        W = crgb.World(w)
        keep.append(W)
        specs.append(crgb.ProblemSpec(W, pr.q_start, pr.goal, H, seeds=seeds))
        probs.append((W, pr, seeds))
    p = dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE) if ik else None
    n_p, iters_p = 8, 2
    V = sum(sd.size for _, _, sd in probs)
    g = torch.Generator(device="cuda").manual_seed(5)
    eps = torch.randn(iters_p * n_p * V, device="cuda", generator=g)
    cfg = dict(iters=iters_p, n_particles=n_p, beta=1000.0, k_mu=0.9, k_sigma=0.9, sigma0=0.01, eps=eps)
    out = crgb.solve(ctx, R, specs, p, iters=5, particles=cfg)
    out0 = crgb.solve(ctx, R, specs, p, iters=0, particles=cfg)
    torch.cuda.synchronize()
    # the same particle iterations problem by problem
    means = []
    off = 0
    for (W, pr, sd), spec in zip(probs, specs):
        B, H, D = sd.shape
        mu = torch.tensor(sd, dtype=torch.float32, device="cuda").contiguous()
        sigma = torch.full_like(mu, 0.01)
        for k in range(iters_p):
            e = eps[k * n_p * V + off * n_p: k * n_p * V + (off + sd.size) * n_p].view(B, n_p, H, D)
            crgb.particle_step(R, crgb.ProblemSpec(W, pr.q_start, pr.goal, H), mu, sigma, e.contiguous(), p,
                               beta=1000.0, k_mu=0.9, k_sigma=0.9)
        means.append(mu)
        off += sd.size
    ref = crgb.solve(ctx, R, specs, p, iters=5, device_seeds=means)
    torch.cuda.synchronize()
    for a, b, m in zip(out, ref, means):
        for k in ("traj", "cost", "cfree", "best", "status"):
            assert torch.equal(getattr(a, k), getattr(b, k)), k
    for a, m in zip(out0, means):   # no L-BFGS iteration: the means themselves
        assert torch.equal(a.traj, m)
