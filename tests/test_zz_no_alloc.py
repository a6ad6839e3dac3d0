"""The evaluation entry point that allocates no device memory.

It exists for callers that cannot let a library allocate: a robot
controller's real-time loop that must not call cudaMalloc/cudaFree once it
runs (those calls take unbounded time and synchronise the device), or an
application whose own pool owns all device memory.  Its scratch lives in a
fixed device array inside the library; the caller passes inputs and outputs.

Checked here through the C ABI: two calls in a row give what the regular
per-problem entry point (cr_eval) gives, within the parity tests' tolerance,
and batches beyond the stated maximum are refused with a clear error.
This file is collected last on purpose.
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


def _close(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.allclose(a, b, rtol=1e-5, atol=1e-6)


def test_noalloc_matches_regular_entry_point_twice(setup):
    R, cases = setup
    ref = [crgb.evaluate(R, spec, th) for _, spec, th in cases]
    for call in range(2):
        out = crgb.evaluate_batch_noalloc(R, [c[1] for c in cases], [c[2] for c in cases])
        torch.cuda.synchronize()
        for r, o in zip(ref, out):
            assert _close(o["cost"], r["cost"]), call
            assert _close(o["grad"], r["grad"]), call
            assert _close(o["terms"], r["terms"]), call
            assert torch.equal(o["cfree"], r["cfree"]), call


def test_noalloc_refuses_oversized_batches(setup):
    R, cases = setup
    W, spec, th = cases[0]
    with pytest.raises(crgb.CrError, match="CR_NOALLOC_MAX_PROBLEMS"):
        crgb.evaluate_batch_noalloc(R, [spec] * 257, [th[:1]] * 257)
    # one problem with more tiles than the scratch tables hold
    big = torch.zeros((40000, 32, R.dof), device="cuda")
    with pytest.raises(crgb.CrError, match="CR_NOALLOC_MAX_TILES"):
        crgb.evaluate_batch_noalloc(R, [spec], [big])
