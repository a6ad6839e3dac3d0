"""The evaluation entry point that allocates no device memory.

It exists for callers that cannot let a library allocate: a robot
controller's real-time loop that must not call cudaMalloc/cudaFree once it
runs (those calls take unbounded time and synchronise the device), or an
application whose own pool owns all device memory.  Its scratch lives in a
fixed device array inside the library; the caller passes inputs and outputs.

Checked here through the C ABI: two calls in a row give what the regular
per-problem entry point (cr_eval) gives, bit for bit (trajectory problems and
IK-mode problems of uneven trajectory counts), batches beyond the stated
maximum are refused with a clear error, and a call on a stream that is being
captured is refused before it enqueues anything.  This file is collected last
on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2310_17274_gb300 import crgb, synth

from scenes import line_search_batch, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_2310_17274_gb300 import build
    build.build_library()
    assert torch.cuda.is_available()
    rb = scene(spheres=synth.SPHERES_60)[0]
    R = crgb.Robot(rb)
    cases = []
    for k, (K, B, H, alphas) in enumerate([(8, 4, 32, (0.01, 0.3, 0.7, 1.0)), (70, 4, 48, (0.1, 0.9)),
                                           (20, 50, 1, (1.0,))]):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=K, n_seeds=B, horizon=H,
                         world_seed=30 + k, problem_seed=40 + k)
        theta = line_search_batch(pr, np.random.default_rng(k), alphas=alphas)
        W = crgb.World(w)
        spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H)
        cases.append((W, spec, torch.tensor(theta, dtype=torch.float32, device="cuda")))
    return R, cases


def _same(ref, out, call):
    for r, o in zip(ref, out):
        for k in ("cost", "grad", "terms", "cfree"):
            assert torch.equal(o[k], r[k]), (call, k)


def test_noalloc_matches_regular_entry_point_twice(setup):
    R, cases = setup
    ref = [crgb.evaluate(R, spec, th) for _, spec, th in cases]
    for call in range(2):
        out = crgb.evaluate_batch_noalloc(R, [c[1] for c in cases], [c[2] for c in cases])
        torch.cuda.synchronize()
        _same(ref, out, call)


def test_noalloc_ik_mode_uneven_problems_twice(setup):
    """IK mode (single states on their own kernel): problems of 1, 37, 64 and
    300 configurations with different worlds in one call."""
    R, _ = setup
    rb = scene(spheres=synth.SPHERES_60)[0]
    specs, thetas = [], []
    rng = np.random.default_rng(50)
    for k, (K, n) in enumerate([(0, 1), (40, 37), (12, 64), (70, 300)]):
        _, w, pr = scene(spheres=synth.SPHERES_60, n_boxes=K, n_seeds=1, horizon=1, world_seed=60 + k,
                         problem_seed=70 + k)
        W = crgb.World(w)
        specs.append((W, crgb.ProblemSpec(W, pr.q_start, pr.goal, 1)))
        q = synth.uniform_config(rng, rb, n)[:, None, :]
        thetas.append(torch.tensor(q, dtype=torch.float32, device="cuda"))
    p = dict(flags=crgb.IK_MODE | crgb.SELF)
    ref = [crgb.evaluate(R, sp, th, p) for (_, sp), th in zip(specs, thetas)]
    for call in range(2):
        out = crgb.evaluate_batch_noalloc(R, [sp for _, sp in specs], thetas, p)
        torch.cuda.synchronize()
        _same(ref, out, call)
    assert 0 < int(sum(int(r["cfree"].sum()) for r in ref)) < 402


def test_noalloc_refuses_a_capturing_stream(setup):
    R, cases = setup
    _, spec, th = cases[0]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with pytest.raises(crgb.CrError, match="captured"):
        with torch.cuda.graph(g, stream=s):
            crgb.evaluate_batch_noalloc(R, [spec], [th])
    torch.cuda.synchronize()
    # the library is usable afterwards
    out = crgb.evaluate_batch_noalloc(R, [spec], [th])
    ref = crgb.evaluate(R, spec, th)
    torch.cuda.synchronize()
    _same([ref], out, 0)


def test_noalloc_refuses_oversized_batches(setup):
    R, cases = setup
    W, spec, th = cases[0]
    with pytest.raises(crgb.CrError, match="CR_NOALLOC_MAX_PROBLEMS"):
        crgb.evaluate_batch_noalloc(R, [spec] * 257, [th[:1]] * 257)
    # one problem with more tiles than the scratch tables hold
    big = torch.zeros((40000, 32, R.dof), device="cuda")
    with pytest.raises(crgb.CrError, match="CR_NOALLOC_MAX_TILES"):
        crgb.evaluate_batch_noalloc(R, [spec], [big])
