"""Step-wise GPU parity of the L-BFGS step and the line-search selection
against the FP64 oracle (the same float32-rounded state fed to both).

Bars: direction and candidates ||d|| <= 1e-3 ||ref||; chosen index equal
unless the oracle's Armijo/Wolfe margin is within 1e-4 |c_0|; new iterate
equal to the chosen candidate.
"""
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


def _history_state(n, m, k_steps, seed):
    """An oracle L-BFGS state after k_steps steps on a mildly non-quadratic
    function, rounded to float32."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n)) / np.sqrt(n)
    A = A @ A.T + np.eye(n)
    st = oracle.LbfgsState(n, m)
    x = rng.normal(size=n)
    for _ in range(k_steps):
        st.x[:] = x
        st.g[:] = A @ x + 0.3 * np.sin(3 * x)
        d = st.direction()
        x = x + 0.4 * d
    st.x[:] = x
    st.g[:] = A @ x + 0.3 * np.sin(3 * x)
    for name in ("x", "g", "x_prev", "g_prev", "s", "y", "rho"):
        setattr(st, name, f32(getattr(st, name)))
    return st


def _ring(a, it):
    """Oracle history (oldest first, newest last) as the device ring holds it
    when iter = it: logical pair i in slot (it - 1 + i) mod m."""
    return np.roll(a, (int(it) - 1) % a.shape[0], axis=0)


def _load(buf, b, st):
    buf.x[b] = torch.tensor(st.x, dtype=torch.float32)
    buf.g[b] = torch.tensor(st.g, dtype=torch.float32)
    buf.x_prev[b] = torch.tensor(st.x_prev, dtype=torch.float32)
    buf.g_prev[b] = torch.tensor(st.g_prev, dtype=torch.float32)
    it = int(st.iter[0])
    buf.s[b] = torch.tensor(_ring(st.s, it), dtype=torch.float32)
    buf.y[b] = torch.tensor(_ring(st.y, it), dtype=torch.float32)
    buf.rho[b] = torch.tensor(_ring(st.rho, it), dtype=torch.float32)
    buf.iter[b] = it


@pytest.mark.parametrize("H,m,k_steps", [(32, 6, 0), (32, 6, 1), (32, 6, 3), (48, 6, 9),
                                         (1, 6, 4), (64, 16, 20)])
def test_propose_matches_oracle(H, m, k_steps):
    rb, _, _ = scene()
    D = rb.dof
    n = H * D
    B = 3
    alphas = list(synth.ALPHA_8)
    p = dict(history=m, alpha=alphas)
    buf = crgb.OptBuffers(B, H, D, m, len(alphas), device="cuda")
    refs = []
    for b in range(B):
        st = _history_state(n, m, k_steps, seed=100 * b + H + k_steps)
        # keep x inside the joint limits so clipping is exercised only at the edges
        lo, hi = np.tile(rb.q_lo, H), np.tile(rb.q_hi, H)
        st.x[:] = f32(np.clip(st.x, lo * 0.9, hi * 0.9))
        _load(buf, b, st)
        d = st.direction()
        cand = oracle.ls_candidates(p, st.x, d, rb.q_lo, rb.q_hi, D)
        refs.append((d, cand, st))
    R = crgb.Robot(rb)
    crgb.opt_propose(R, p, buf)
    torch.cuda.synchronize()
    for b, (d, cand, st) in enumerate(refs):
        dg = buf.dir[b].cpu().numpy()
        assert np.linalg.norm(dg - d) <= 1e-3 * np.linalg.norm(d) + 1e-7, (b, np.linalg.norm(dg - d))
        cg = buf.cand[b].cpu().numpy()
        assert np.abs(cg - cand).max() <= 1e-3 * np.abs(d).max() + 1e-6
        it = int(st.iter[0])
        np.testing.assert_allclose(buf.s[b].cpu().numpy(), _ring(st.s, it), atol=1e-6)
        np.testing.assert_allclose(buf.y[b].cpu().numpy(), _ring(st.y, it), atol=1e-5, rtol=1e-5)
        np.testing.assert_allclose(buf.rho[b].cpu().numpy(), _ring(st.rho, it), rtol=1e-4)
        np.testing.assert_array_equal(buf.x_prev[b].cpu().numpy(), st.x.astype(np.float32))
        assert int(buf.iter[b]) == int(st.iter[0])


_EVAL_FLAGS = crgb.SWEPT | crgb.SPEED | crgb.SELF

# line-search variants of Sec. 7.3: (step sizes, selection flags, seeds that must
# be decided away from every threshold)
LS_VARIANTS = {
    "noisy-ls": ([0.01, 0.3, 0.7, 1.0], crgb.WOLFE, 4),
    "noisy-ls-1": ([0.01, 1.0], crgb.WOLFE, 4),
    "strong-wolfe": ([0.01, 0.3, 0.7, 1.0], crgb.WOLFE | crgb.STRONG_WOLFE, 3),
    "armijo-only": ([0.01, 0.3, 0.7, 1.0], 0, 4),
    "no-ls": ([1.0], 0, 6),
}


@pytest.mark.parametrize("variant", list(LS_VARIANTS))
def test_select_matches_oracle_on_real_problem(variant):
    """Propose from evaluated seeds, evaluate the candidates with the oracle,
    then select on both sides, for each line-search variant of Sec. 7.3."""
    rb, w, pr = scene(n_seeds=6, horizon=32)
    D, H, B = rb.dof, 32, 6
    n = H * D
    alphas, ls_flags, min_strict = LS_VARIANTS[variant]
    p = dict(alpha=alphas, flags=_EVAL_FLAGS | ls_flags)
    na = len(alphas)
    ev0 = oracle.evaluate(rb, w, pr.q_start, pr.goal, pr.seeds)
    buf = crgb.OptBuffers(B, H, D, 6, na, device="cuda")
    buf.x.copy_(torch.tensor(pr.seeds.reshape(B, n), dtype=torch.float32))
    buf.g.copy_(torch.tensor(f32(ev0["grad"]).reshape(B, n), dtype=torch.float32))
    buf.c.copy_(torch.tensor(f32(ev0["cost"]), dtype=torch.float32))
    buf.best_c.fill_(float("inf"))
    R = crgb.Robot(rb)
    crgb.opt_propose(R, p, buf)
    torch.cuda.synchronize()
    cand = f32(buf.cand.cpu().numpy())
    d = f32(buf.dir.cpu().numpy())
    ev = oracle.evaluate(rb, w, pr.q_start, pr.goal, cand.reshape(B * na, H, D))
    cc = f32(ev["cost"]).reshape(B, na)
    cgr = f32(ev["grad"]).reshape(B, na, n)
    buf.cand_cost.copy_(torch.tensor(cc, dtype=torch.float32))
    buf.cand_grad.copy_(torch.tensor(cgr, dtype=torch.float32))
    buf.cand_cfree.copy_(torch.tensor(ev["cfree"].reshape(B, na).astype(np.uint8)))
    crgb.opt_select(R, p, buf)
    torch.cuda.synchronize()
    idx_g = buf.ls_index.cpu().numpy()
    n_strict = 0
    for b in range(B):
        idx, margin = oracle.ls_select(p, f32(ev0["cost"])[b], f32(ev0["grad"]).reshape(B, n)[b],
                                       d[b], cc[b], cgr[b])
        if margin >= 1e-4 * abs(ev0["cost"][b]):
            n_strict += 1
            assert idx_g[b] == idx, (b, idx_g[b], idx)
        k = idx_g[b]
        np.testing.assert_array_equal(buf.x[b].cpu().numpy(), cand[b, k].astype(np.float32))
        np.testing.assert_array_equal(buf.g[b].cpu().numpy(), cgr[b, k].astype(np.float32))
        assert float(buf.c[b]) == np.float32(cc[b, k])
        assert float(buf.best_c[b]) == np.float32(cc[b, k])  # best was +inf
        np.testing.assert_array_equal(buf.best_x[b].cpu().numpy(), cand[b, k].astype(np.float32))
    assert n_strict >= min_strict


def test_weak_and_strong_wolfe_choose_differently():
    """Directional derivatives g_l . d of -0.95, -0.5, +0.5 and +0.95 times
    |g_0 . d| with every candidate below the Armijo line: the weak Wolfe test
    (g_l . d >= 0.9 g_0 . d) passes steps 1-3 and takes 3, the strong one
    (|g_l . d| <= 0.9 |g_0 . d|) passes 1-2 and takes 2, Armijo alone takes 3;
    the oracle agrees on each."""
    rb, _, _ = scene()
    D, H, na = rb.dof, 2, 4
    n = H * D
    R = crgb.Robot(rb)
    g0 = np.zeros(n, np.float32)
    g0[0] = 1.0                                   # g_0 . d = -1 with d = -g_0
    d = -g0
    slopes = np.array([-0.95, -0.5, 0.5, 0.95], np.float32)
    cgrad = np.zeros((na, n), np.float32)
    cgrad[:, 0] = -slopes                         # g_l . d = slopes[l]
    cost = np.full(na, 0.5, np.float32)           # c_0 = 1: Armijo holds for every step
    expect = {crgb.WOLFE: 3, crgb.WOLFE | crgb.STRONG_WOLFE: 2, 0: 3}
    for fl, want in expect.items():
        p = dict(alpha=[0.1, 0.3, 0.7, 1.0], flags=_EVAL_FLAGS | fl)
        buf = crgb.OptBuffers(1, H, D, 2, na, device="cuda")
        buf.x.zero_()
        buf.g.copy_(torch.tensor(g0)[None])
        buf.dir.copy_(torch.tensor(d)[None])
        buf.c.fill_(1.0)
        buf.best_c.fill_(float("inf"))
        buf.cand.copy_(torch.arange(na, dtype=torch.float32).view(1, na, 1).expand(1, na, n))
        buf.cand_cost.copy_(torch.tensor(cost)[None])
        buf.cand_grad.copy_(torch.tensor(cgrad)[None])
        buf.cand_cfree.fill_(1)
        crgb.opt_select(R, p, buf)
        torch.cuda.synchronize()
        idx, _ = oracle.ls_select(p, 1.0, g0, d, cost, cgrad)
        assert idx == want, (fl, idx)
        assert int(buf.ls_index[0]) == want, (fl, int(buf.ls_index[0]))
        assert float(buf.x[0, 0]) == float(want)


def test_select_fallback_and_best_tracking():
    """No candidate passes: index 0 is taken; a worse cost leaves the best alone."""
    rb, _, _ = scene()
    D, H, B, na = rb.dof, 4, 2, 3
    n = H * D
    p = dict(alpha=[0.01, 0.5, 1.0], flags=0)
    buf = crgb.OptBuffers(B, H, D, 2, na, device="cuda")
    rng = np.random.default_rng(0)
    buf.x.copy_(torch.tensor(rng.normal(size=(B, n)), dtype=torch.float32))
    buf.g.copy_(torch.tensor(rng.normal(size=(B, n)), dtype=torch.float32))
    buf.dir.copy_(-buf.g)
    buf.c.fill_(1.0)
    buf.best_c.copy_(torch.tensor([0.5, 10.0]))
    buf.best_x.fill_(7.0)
    buf.cand.copy_(torch.tensor(rng.normal(size=(B, na, n)), dtype=torch.float32))
    buf.cand_cost.fill_(2.0)                      # all worse than c = 1: Armijo fails
    buf.cand_grad.zero_()
    buf.cand_cfree.fill_(1)
    R = crgb.Robot(rb)
    crgb.opt_select(R, p, buf)
    torch.cuda.synchronize()
    assert buf.ls_index.cpu().tolist() == [0, 0]
    np.testing.assert_array_equal(buf.x.cpu().numpy(), buf.cand[:, 0].cpu().numpy())
    assert float(buf.best_c[0]) == 0.5 and float(buf.best_x[0, 0]) == 7.0     # kept
    assert float(buf.best_c[1]) == 2.0                                         # improved on 10
    np.testing.assert_array_equal(buf.best_x[1].cpu().numpy(), buf.cand[1, 0].cpu().numpy())
    assert int(buf.best_cfree[1]) == 1
    # NaN candidate never becomes the best
    buf.cand_cost.fill_(float("nan"))
    buf.c.fill_(1.0)
    crgb.opt_select(R, p, buf)
    torch.cuda.synchronize()
    assert float(buf.best_c[0]) == 0.5
