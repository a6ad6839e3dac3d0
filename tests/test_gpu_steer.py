"""Parallel steering (Sec. 5, Alg. "Parallel Steering") through cr_steer
against the oracle: per-sample validity flags bit-exact away from the
clearance threshold, and per edge the last valid sample, the new vertex and
its distance."""
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


def _edges(rb, rng, E):
    a = synth.uniform_config(rng, rb, E)
    b = np.clip(a + rng.normal(0, 0.6, size=a.shape), rb.q_lo, rb.q_hi)
    return f32(np.stack([a, b], axis=1))


@pytest.mark.parametrize("n_boxes", [0, 16])
def test_steer_matches_oracle(n_boxes):
    rb, w, _ = scene(spheres=synth.SPHERES_60, n_boxes=max(n_boxes, 1), world_seed=9)
    if n_boxes == 0:
        w = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    rng = np.random.default_rng(11)
    edges = _edges(rb, rng, 120)
    ed = torch.tensor(edges, dtype=torch.float32, device="cuda")
    n = crgb.steer_steps(ed, 0.05)
    assert n == oracle.steer_steps(edges, 0.05)
    R, W = crgb.Robot(rb), crgb.World(w)
    out = crgb.steer(R, W, ed, n)
    torch.cuda.synchronize()
    last = out["last"].cpu().numpy()
    valid = out["valid"].cpu().numpy().astype(bool)
    v_new = out["v_new"].cpu().numpy()
    dist = out["dist"].cpu().numpy()
    # the GPU's own flags decide its answer
    for e in range(len(edges)):
        bad = np.flatnonzero(~valid[e])
        assert last[e] == (bad[0] - 1 if len(bad) else n)
    # flags against the oracle's discrete test on the same float32 samples
    q = np.stack([edges[:, 0] + (i / n) * (edges[:, 1] - edges[:, 0]) for i in range(n + 1)], axis=1)
    samples = f32(q).reshape(-1, 1, rb.dof)
    p = dict(flags=oracle.IK_MODE | oracle.SELF)
    ref = oracle.evaluate(rb, w, samples[0, 0], np.array([0, 0, 0, 1.0, 0, 0, 0]), samples, p,
                          want_grad=False)
    ok = ref["margin"] >= 1e-5
    flat = valid.reshape(-1)
    assert np.array_equal(flat[ok], ref["cfree"][ok])
    # per edge against the oracle's steering wherever no sample is near a threshold
    o_last, o_v, o_d = oracle.steer(rb, w, edges, n)
    near = (~ok).reshape(len(edges), n + 1).any(axis=1)
    assert (~near).sum() >= len(edges) // 2
    assert np.array_equal(last[~near], o_last[~near])
    np.testing.assert_allclose(v_new[~near], o_v[~near], atol=2e-6)
    np.testing.assert_allclose(dist[~near], o_d[~near], rtol=1e-5, atol=2e-6)
    # both outcomes occur (random configurations also collide with the robot itself)
    assert (last < n).any() and (last == n).any()


def test_steer_start_in_collision_and_empty():
    rb, _, _ = scene()
    a = np.zeros(rb.dof)
    _, sp, _ = oracle.fk(rb, a)
    w = synth.World(pose=f32(np.array([[*sp[10, :3], 1.0, 0.0, 0.0, 0.0]])), half_ext=f32(np.full((1, 3), 0.05)))
    R, W = crgb.Robot(rb), crgb.World(w)
    ed = torch.tensor(np.stack([a, np.full(rb.dof, 0.3)])[None], dtype=torch.float32, device="cuda")
    out = crgb.steer(R, W, ed, 5)
    torch.cuda.synchronize()
    assert int(out["last"][0]) == -1
    assert torch.equal(out["v_new"][0], ed[0, 0]) and float(out["dist"][0]) == 0.0
    empty = crgb.steer(R, W, torch.zeros((0, 2, rb.dof), device="cuda"), 4)
    assert empty["last"].numel() == 0
