"""Pins of the FP64 oracle against things other than itself: values the paper
prints, closed forms, invariants, brute force and finite differences.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2310_17274_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers (independent of the oracle's code)
# ---------------------------------------------------------------------------

def _mat4(tf12):
    T = np.eye(4)
    T[:3, :] = np.asarray(tf12).reshape(3, 4)
    return T


def _robot(spheres=synth.SPHERES_42, seed=0):
    return synth.make_robot(spheres, seed=seed)


def _chain(n_joints, axes=None, spheres_per_link=2, seed=5):
    """A short chain for finite-difference pins."""
    axes = axes or [2, 1, 0, 2, 1, 0, 2][:n_joints]
    rb = synth.make_robot(tuple([spheres_per_link] * n_joints), seed=seed, axes=tuple(axes))
    return rb


def _quat_axis_angle(axis, ang):
    axis = np.asarray(axis, dtype=float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])


# ---------------------------------------------------------------------------
# constants the paper states
# ---------------------------------------------------------------------------

def test_default_constants_match_paper(oracle_mod):
    p = oracle_mod.params_default()
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            name, value = line.split()[:2]
            if name == "alpha":
                assert p["alpha"] == [float(v) for v in value.split(",")]
            else:
                assert p[name] == pytest.approx(float(value), rel=0, abs=0), name


# ---------------------------------------------------------------------------
# forward kinematics (Sec. 3.1, App. E.1 Table "Joint Transformation matrices")
# ---------------------------------------------------------------------------

def test_joint_axes_match_table(oracle_mod):
    """One joint with F = I at theta = pi/2 moves unit points as the table's
    revolute matrices do."""
    with open(os.path.join(GOLDEN, "joint_transform_axes.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for ax, *vals in rows:
        a = "xyz".index(ax)
        inp = np.array(vals[:3], dtype=float)
        exp = np.array(vals[3:], dtype=float)
        ident = np.eye(3, 4).reshape(12)
        rb = synth.Robot(fixed_tf=np.stack([ident, ident]), axis=np.array([a], np.int32),
                         q_lo=np.array([-3.0]), q_hi=np.array([3.0]), v_max=np.ones(1),
                         a_max=np.ones(1), j_max=np.ones(1),
                         spheres=np.array([[*inp, 0.1]]), sphere_link=np.array([0], np.int32),
                         pairs=np.zeros((0, 2), np.int32))
        _, sp, _ = oracle_mod.fk(rb, [math.pi / 2])
        np.testing.assert_allclose(sp[0, :3], exp, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_full_link_transformation_matches_table(oracle_mod, axis):
    """Right-hand column of the table: F * J(theta) written entrywise with
    f_0..f_11 (the X row's (3,3) entry read as f_10 cos, the printed
    "f_10 sin" being a typo)."""
    rng = np.random.default_rng(axis)
    f = rng.normal(size=12)
    th = 0.7
    c, s = math.cos(th), math.sin(th)
    if axis == 0:
        exp = [f[0], f[1] * c + f[2] * s, -f[1] * s + f[2] * c, f[3],
               f[4], f[5] * c + f[6] * s, -f[5] * s + f[6] * c, f[7],
               f[8], f[9] * c + f[10] * s, -f[9] * s + f[10] * c, f[11]]
    elif axis == 1:
        exp = [f[0] * c - f[2] * s, f[1], f[0] * s + f[2] * c, f[3],
               f[4] * c - f[6] * s, f[5], f[4] * s + f[6] * c, f[7],
               f[8] * c - f[10] * s, f[9], f[8] * s + f[10] * c, f[11]]
    else:
        exp = [f[0] * c + f[1] * s, -f[0] * s + f[1] * c, f[2], f[3],
               f[4] * c + f[5] * s, -f[4] * s + f[5] * c, f[6], f[7],
               f[8] * c + f[9] * s, -f[8] * s + f[9] * c, f[10], f[11]]
    ident = np.eye(3, 4).reshape(12)
    rb = synth.Robot(fixed_tf=np.stack([f, ident]), axis=np.array([axis], np.int32),
                     q_lo=np.array([-3.0]), q_hi=np.array([3.0]), v_max=np.ones(1),
                     a_max=np.ones(1), j_max=np.ones(1), spheres=np.zeros((0, 4)),
                     sphere_link=np.zeros(0, np.int32), pairs=np.zeros((0, 2), np.int32))
    lt, _, _ = oracle_mod.fk(rb, [th])
    np.testing.assert_allclose(lt[0], exp, atol=1e-14)


def test_fk_zero_configuration_is_composed_fixed_transforms(oracle_mod):
    rb = _robot()
    lt, sp, ee = oracle_mod.fk(rb, np.zeros(rb.dof))
    T = np.eye(4)
    for j in range(rb.dof):
        T = T @ _mat4(rb.fixed_tf[j])
        np.testing.assert_allclose(lt[j], T[:3].reshape(12), atol=1e-14)
    np.testing.assert_allclose(ee, (T @ _mat4(rb.fixed_tf[rb.dof]))[:3].reshape(12), atol=1e-14)
    for i in range(rb.n_spheres):
        Tl = np.eye(4)
        for j in range(rb.sphere_link[i] + 1):
            Tl = Tl @ _mat4(rb.fixed_tf[j])
        np.testing.assert_allclose(sp[i, :3], (Tl @ np.r_[rb.spheres[i, :3], 1])[:3], atol=1e-14)
        assert sp[i, 3] == rb.spheres[i, 3]


def test_fk_rigidity_and_orthonormality(oracle_mod):
    rb = _robot()
    rng = np.random.default_rng(1)
    _, sp0, _ = oracle_mod.fk(rb, np.zeros(rb.dof))
    for _ in range(5):
        q = synth.uniform_config(rng, rb)
        lt, sp, ee = oracle_mod.fk(rb, q)
        for T in list(lt) + [ee]:
            R = np.asarray(T).reshape(3, 4)[:, :3]
            assert np.abs(R.T @ R - np.eye(3)).max() < 1e-12
            assert abs(np.linalg.det(R) - 1) < 1e-12
        for l in range(rb.dof):
            idx = np.where(rb.sphere_link == l)[0]
            d0 = np.linalg.norm(sp0[idx, None, :3] - sp0[None, idx, :3], axis=-1)
            d1 = np.linalg.norm(sp[idx, None, :3] - sp[None, idx, :3], axis=-1)
            np.testing.assert_allclose(d0, d1, atol=1e-12)


def test_fk_first_joint_rotation_is_rigid_about_base_axis(oracle_mod):
    """Turning joint 0 (a z joint at the base) by phi rotates every sphere
    about the world z axis by phi."""
    rb = _robot()
    rng = np.random.default_rng(3)
    q = synth.uniform_config(rng, rb) * 0.5
    _, sp, _ = oracle_mod.fk(rb, q)
    q2 = q.copy()
    q2[0] += 0.4
    _, sp2, _ = oracle_mod.fk(rb, q2)
    c, s = math.cos(0.4), math.sin(0.4)
    Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    np.testing.assert_allclose(sp2[:, :3], sp[:, :3] @ Rz.T, atol=1e-12)


# ---------------------------------------------------------------------------
# box signed distance (Sec. 3.5)
# ---------------------------------------------------------------------------

def _box(seed=0):
    rng = np.random.default_rng(seed)
    pose = np.concatenate([rng.uniform(-0.5, 0.5, 3),
                           _quat_axis_angle(rng.normal(size=3), rng.uniform(0, 3))])
    he = rng.uniform(0.05, 0.3, 3)
    return pose, he


def _rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_sphere_at_box_centre(oracle_mod):
    """Sphere-in-box distance at the centre = -(min half-extent gap + radius)."""
    for seed in range(4):
        pose, he = _box(seed)
        phi, _ = oracle_mod.box_sdf(pose, he, pose[:3])
        r = 0.05
        assert phi - r == pytest.approx(-(he.min() + r), abs=1e-14)


def test_box_face_and_corner_regions(oracle_mod):
    pose, he = _box(7)
    R = _rot(pose[3:])
    # face region along local +y
    u = np.array([0.3 * he[0], he[1] + 0.17, -0.2 * he[2]])
    phi, g = oracle_mod.box_sdf(pose, he, pose[:3] + R @ u)
    assert phi == pytest.approx(0.17, abs=1e-12)
    np.testing.assert_allclose(g, R[:, 1], atol=1e-12)
    # corner region
    u = he * np.array([1, -1, 1]) + np.array([0.1, -0.2, 0.05])
    phi, g = oracle_mod.box_sdf(pose, he, pose[:3] + R @ u)
    assert phi == pytest.approx(math.sqrt(0.1 ** 2 + 0.2 ** 2 + 0.05 ** 2), abs=1e-12)
    # inside, closest to local -x face
    u = np.array([-he[0] + 0.01, 0.0, 0.0])
    if he[0] - 0.01 < min(he[1], he[2]):
        phi, g = oracle_mod.box_sdf(pose, he, pose[:3] + R @ u)
        assert phi == pytest.approx(-0.01, abs=1e-12)
        np.testing.assert_allclose(g, -R[:, 0], atol=1e-12)


def test_box_sdf_brute_force(oracle_mod):
    """Distance to a densely sampled box surface (minus inside)."""
    pose, he = _box(3)
    R = _rot(pose[3:])
    n = 60
    grids = []
    lin = [np.linspace(-h, h, n) for h in he]
    for a in range(3):
        for sgn in (-1, 1):
            b, c = [k for k in range(3) if k != a]
            B, Cc = np.meshgrid(lin[b], lin[c], indexing="ij")
            P = np.zeros((n * n, 3))
            P[:, a] = sgn * he[a]
            P[:, b] = B.ravel()
            P[:, c] = Cc.ravel()
            grids.append(P)
    surf = np.concatenate(grids)
    step = 2 * he.max() / (n - 1)
    rng = np.random.default_rng(0)
    for _ in range(40):
        u = rng.uniform(-1.8, 1.8, 3) * he
        inside = np.all(np.abs(u) <= he)
        d = np.linalg.norm(surf - u, axis=1).min()
        phi, g = oracle_mod.box_sdf(pose, he, pose[:3] + R @ u)
        exp = -d if inside else d
        assert abs(phi - exp) <= step, (u, phi, exp)
        # gradient = finite difference of the distance
        for a in range(3):
            e = np.zeros(3)
            e[a] = 1e-6
            p1, _ = oracle_mod.box_sdf(pose, he, pose[:3] + R @ u + e)
            p0, _ = oracle_mod.box_sdf(pose, he, pose[:3] + R @ u - e)
            assert (p1 - p0) / 2e-6 == pytest.approx(g[a], abs=1e-6)


# ---------------------------------------------------------------------------
# Eq. 10 and Eq. 17: continuity and slopes
# ---------------------------------------------------------------------------

def test_smooth_distance_profile(oracle_mod):
    eta = 0.025
    for d in [-0.1, -eta - 1e-3, -0.02, -0.01, -1e-9, 0.0, 1e-9, 0.01, 0.3]:
        v, s = oracle_mod.smooth_distance(d, eta)
        vp, _ = oracle_mod.smooth_distance(d + 1e-7, eta)
        vm, _ = oracle_mod.smooth_distance(d - 1e-7, eta)
        assert (vp - vm) / 2e-7 == pytest.approx(s, abs=2e-6)
    # continuity of value and slope at 0 and -eta; values fixed by Eq. 10
    assert oracle_mod.smooth_distance(0.0, eta)[0] == pytest.approx(0.5 * eta)
    assert oracle_mod.smooth_distance(1e-12, eta)[0] == pytest.approx(0.5 * eta)
    assert oracle_mod.smooth_distance(-eta, eta) == (0.0, 0.0)
    assert oracle_mod.smooth_distance(0.2, eta) == (0.2 + 0.5 * eta, 1.0)
    assert oracle_mod.smooth_distance(-eta / 2, eta)[0] == pytest.approx(0.5 / eta * (eta / 2) ** 2)


def test_bound_cost_profile(oracle_mod):
    lo, hi, e2 = -1.0, 2.0, 0.1
    assert oracle_mod.bound_cost(lo, lo, hi, e2)[0] == pytest.approx(0.5 * e2)
    assert oracle_mod.bound_cost(hi, lo, hi, e2)[0] == pytest.approx(0.5 * e2)
    assert oracle_mod.bound_cost(0.5, lo, hi, e2) == (0.0, 0.0)
    assert oracle_mod.bound_cost(lo - 0.3, lo, hi, e2)[0] == pytest.approx(0.3 + 0.05)
    assert oracle_mod.bound_cost(hi + 0.3, lo, hi, e2)[0] == pytest.approx(0.3 + 0.05)
    assert oracle_mod.bound_cost(lo + e2, lo, hi, e2)[0] == pytest.approx(0.0, abs=1e-15)
    for q in np.linspace(lo - 0.2, hi + 0.2, 97):
        v, s = oracle_mod.bound_cost(q, lo, hi, e2)
        vp, _ = oracle_mod.bound_cost(q + 1e-7, lo, hi, e2)
        vm, _ = oracle_mod.bound_cost(q - 1e-7, lo, hi, e2)
        assert (vp - vm) / 2e-7 == pytest.approx(s, abs=1e-5)
        # symmetric profile about the middle of the range
        vs, _ = oracle_mod.bound_cost(lo + hi - q, lo, hi, e2)
        assert v == pytest.approx(vs, abs=1e-12)


# ---------------------------------------------------------------------------
# App. A.5 five-point stencils
# ---------------------------------------------------------------------------

def test_stencils_exact_on_polynomials(oracle_mod):
    dt = 0.05
    H = 20
    ts = np.arange(H + 5) * dt           # ext indices 0..H+4
    p4 = lambda t: 0.3 - 0.2 * t + 0.7 * t ** 2 - 0.4 * t ** 3 + 0.9 * t ** 4
    dp4 = lambda t: -0.2 + 1.4 * t - 1.2 * t ** 2 + 3.6 * t ** 3
    ddp4 = lambda t: 1.4 - 2.4 * t + 10.8 * t ** 2
    p3 = lambda t: 0.1 + 0.5 * t - 0.3 * t ** 2 + 2.0 * t ** 3
    # interior samples only (the padding holds copies, not the polynomial)
    for poly, checks in [(p4, "va"), (p3, "j")]:
        ext = poly(ts)
        q0 = np.array([ext[2]])
        theta = ext[3:H + 3, None]
        v, a, j = oracle_mod.stencil(q0, theta, dt)
        for e in range(4, H + 1):         # samples whose five points are all genuine
            t = ts[e]
            k = e - 2
            if "v" in checks:
                assert v[k, 0] == pytest.approx(dp4(t), rel=1e-9, abs=1e-9)
            if "a" in checks:
                assert a[k, 0] == pytest.approx(ddp4(t), rel=1e-7, abs=1e-7)
            if "j" in checks:
                assert j[k, 0] == pytest.approx(12.0, rel=1e-9)


def test_constant_trajectory_has_zero_derivatives_and_smoothness(oracle_mod):
    rb = _robot()
    q0 = np.linspace(-0.3, 0.3, rb.dof)
    theta = np.tile(q0, (8, 1))
    v, a, j = oracle_mod.stencil(q0, theta, 0.05)
    assert np.abs(v).max() < 1e-12 and np.abs(a).max() < 1e-10 and np.abs(j).max() < 1e-9
    w = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    ee = oracle_mod.goal_pose_from_fk(rb, q0)
    out = oracle_mod.evaluate(rb, w, q0, ee, theta[None])
    assert out["terms"][0, 3] < 1e-12         # smoothness
    assert out["terms"][0, 4] == pytest.approx(0.0, abs=1e-6)  # goal reached


def test_padding_ties_boundary_states(oracle_mod):
    """The first sample sees three copies of the start state, the last sample
    three copies of theta_H: a step from q0 to q1 at t=1 gives the stencil
    values of the step function."""
    dt = 0.1
    q0 = np.array([0.0])
    theta = np.ones((6, 1))
    v, a, j = oracle_mod.stencil(q0, theta, dt)
    # sample e=2 uses [q0, q0, q0, q1, q1]
    assert v[0, 0] == pytest.approx((8 - 1) / (12 * dt))
    assert a[0, 0] == pytest.approx((16 - 1) / (12 * dt * dt))
    assert j[0, 0] == pytest.approx((-2 + 1) / (2 * dt ** 3))
    # last sample e=H+2 uses [q_{H-2}, q_{H-1}, q_H, q_H, q_H] = all ones
    assert v[-1, 0] == 0 and a[-1, 0] == 0 and j[-1, 0] == 0


# ---------------------------------------------------------------------------
# Eq. 9 self-collision
# ---------------------------------------------------------------------------

def _two_sphere_robot(pairs):
    ident = np.eye(3, 4).reshape(12)
    n = 4
    return synth.Robot(fixed_tf=np.stack([ident] * 4), axis=np.array([2, 2, 2], np.int32),
                       q_lo=-np.ones(3), q_hi=np.ones(3), v_max=np.ones(3), a_max=np.ones(3),
                       j_max=np.ones(3), spheres=np.zeros((n, 4)),
                       sphere_link=np.array([0, 2, 0, 2], np.int32),
                       pairs=np.asarray(pairs, np.int32))


def test_self_penetration_two_spheres(oracle_mod):
    rb = _two_sphere_robot([[0, 1]])
    X = np.array([[0.0, 0, 0, 0.1], [0.15, 0.05, 0, 0.08], [5, 5, 5, 0.1], [9, 9, 9, 0.1]])
    pen, arg, g = oracle_mod.self_penetration(rb, X)
    d = math.hypot(0.15, 0.05)
    assert pen == pytest.approx(0.18 - d)
    assert arg == 0
    u = np.array([0.15, 0.05, 0]) / d
    # d pen / d x_i points from i toward j (descent pushes the spheres apart)
    np.testing.assert_allclose(g[0], u, atol=1e-14)
    np.testing.assert_allclose(g[1], -u, atol=1e-14)
    # separated: no penetration, no gradient
    X[1, :3] = [1.0, 0, 0]
    pen, arg, g = oracle_mod.self_penetration(rb, X)
    assert pen == 0.0 and arg == -1 and np.abs(g).max() == 0


def test_self_penetration_max_and_tie(oracle_mod):
    rb = _two_sphere_robot([[0, 1], [2, 3]])
    # exactly representable coordinates, so the tie is exact
    X = np.array([[0.0, 0, 0, 0.1], [0.125, 0, 0, 0.1], [4, 4, 4, 0.1], [4.125, 4, 4, 0.1]])
    pen, arg, _ = oracle_mod.self_penetration(rb, X)
    assert pen == pytest.approx(0.075) and arg == 0        # tie: first in list wins
    X[3, 0] = 4.0625
    pen, arg, _ = oracle_mod.self_penetration(rb, X)
    assert pen == pytest.approx(0.1375) and arg == 1       # max wins
    X[2, 3] = -1.0                                           # disabled sphere
    pen, arg, _ = oracle_mod.self_penetration(rb, X)
    assert arg == 0


# ---------------------------------------------------------------------------
# Sec. 3.4 sweep
# ---------------------------------------------------------------------------

def test_sweep_stationary_reduces_to_discrete(oracle_mod):
    pose, he = _box(11)
    rng = np.random.default_rng(4)
    eta = 0.025
    for _ in range(30):
        x = pose[:3] + rng.uniform(-1.5, 1.5, 3) * he
        r = 0.06
        S, g, _ = oracle_mod.sweep_box(pose, he, r, x, x, x, eta, 4)
        phi, gphi = oracle_mod.box_sdf(pose, he, x)
        dc, slope = oracle_mod.smooth_distance(r - phi, eta)
        assert S == pytest.approx(dc, abs=1e-15)
        np.testing.assert_allclose(g, -slope * gphi, atol=1e-14)


def test_sweep_detects_thin_box_between_free_waypoints(oracle_mod):
    eta, r = 0.025, 0.05
    pose = np.array([0.0, 0, 0, 1, 0, 0, 0])
    he = np.array([0.01, 0.5, 0.5])            # thin wall at x = 0
    x0, x1, x2 = np.array([-0.6, 0, 0]), np.array([-0.3, 0, 0]), np.array([0.3, 0, 0])
    S_disc, _, _ = oracle_mod.sweep_box(pose, he, r, None, x1, None, eta, 4)
    assert S_disc == 0.0                        # waypoint alone is free
    S, g, _ = oracle_mod.sweep_box(pose, he, r, x0, x1, x2, eta, 4)
    assert S > 0.0                              # crossing found by the forward sweep
    assert g[0] > 0                             # cost grows toward the wall: descent pushes back
    # and the backward neighbour alone (moving away) finds nothing
    S_back, _, _ = oracle_mod.sweep_box(pose, he, r, x0, x1, None, eta, 4)
    assert S_back == 0.0


def test_sweep_march_positions(oracle_mod):
    """Hand-traced march toward a face: the waypoint is free (clearance 0.2 -
    r), the first sample lands where the sphere touches, the next ones advance
    by r + eta; the midpoint bound stops the march."""
    eta, r = 0.025, 0.05
    pose = np.array([0.0, 0, 0, 1, 0, 0, 0])
    he = np.array([0.5, 0.5, 0.5])
    x1 = np.array([-0.7, 0, 0])                 # phi = 0.2
    x2 = np.array([-0.7 + 2 * 0.3, 0, 0])       # midpoint 0.3 away
    S, g, _ = oracle_mod.sweep_box(pose, he, r, None, x1, x2, eta, 4)
    # samples at u = 0.15 (phi = 0.05, pen = 0 -> d_c = eta/2), then u = 0.225 (> 0.3? no)
    # u = 0.225: phi = -0.025 inside -> pen = 0.075 -> d_c = 0.075 + eta/2; next u = 0.3 stops
    exp = 0.5 * eta + (0.075 + 0.5 * eta)
    assert S == pytest.approx(exp, abs=1e-12)
    np.testing.assert_allclose(g, [2.0, 0, 0], atol=1e-12)  # two samples, slope 1 each, -grad phi = +x


def test_sweep_gradient_equals_rigid_translation_derivative(oracle_mod):
    """When every sample is in collision the march offsets are fixed (steps of
    r + eta), so translating the three points together moves every sample with
    x1: the surrogate gradient is then the exact derivative."""
    eta, r = 0.025, 0.06
    pose, he = np.array([0.1, -0.2, 0.05, *_quat_axis_angle([1, 2, 3], 0.4)]), np.array([0.4, 0.35, 0.45])
    x1 = pose[:3] + np.array([0.05, 0.02, -0.03])
    x0 = x1 + np.array([-0.2, 0.1, 0.05])
    x2 = x1 + np.array([0.15, -0.1, 0.1])
    S, g, _ = oracle_mod.sweep_box(pose, he, r, x0, x1, x2, eta, 4)
    assert S > 0
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1e-6
        Sp, _, _ = oracle_mod.sweep_box(pose, he, r, x0 + e, x1 + e, x2 + e, eta, 4)
        Sm, _, _ = oracle_mod.sweep_box(pose, he, r, x0 - e, x1 - e, x2 - e, eta, 4)
        assert (Sp - Sm) / 2e-6 == pytest.approx(g[a], rel=1e-6, abs=1e-8)


def test_sweep_stop_margin_counts_only_reachable_samples(oracle_mod):
    """The stop test u >= L of the march is a decision that matters only when
    the sample at u would be in collision.  Toward a face with the first step
    landing exactly at the midpoint, the sample would touch the box: moving the
    neighbour by 1e-9 adds or drops a term of eta / 2, and the margin is ~0.
    Away from the box the same stop test can change nothing and sets no small
    margin."""
    eta, r, d = 0.025, 0.05, 0.1
    pose = np.array([0.0, 0, 0, 1, 0, 0, 0])
    he = np.array([0.5, 0.5, 0.5])
    x1 = np.array([-0.5 - r - d, 0, 0])          # phi - r = d: first step u0 = d
    toward = x1 + np.array([2 * d, 0, 0])       # midpoint L = d: stop exactly at u0
    S0, _, m0 = oracle_mod.sweep_box(pose, he, r, None, x1, toward, eta, 4)
    Sp, _, _ = oracle_mod.sweep_box(pose, he, r, None, x1, toward + [1e-9, 0, 0], eta, 4)
    assert m0 < 1e-12
    assert S0 == 0.0 and Sp == pytest.approx(0.5 * eta, abs=1e-8)   # the sample touches: pen = 0
    away = x1 - np.array([2 * d, 0, 0])
    S1, _, m1 = oracle_mod.sweep_box(pose, he, r, None, x1, away, eta, 4)
    S2, _, _ = oracle_mod.sweep_box(pose, he, r, None, x1, away - [1e-9, 0, 0], eta, 4)
    assert S1 == 0.0 and S2 == 0.0
    # the waypoint's activation test is the closest decision: |(r - phi) + eta| = d - eta
    assert m1 == pytest.approx(d - eta, abs=1e-12)


def _state_scene(oracle_mod, seed=6):
    """42 spheres, 6 boxes near the arm, 3 trajectories of 7 states with the
    joints pushed toward their limits (the chain folds onto itself)."""
    rb = _robot()
    rng = np.random.default_rng(seed)
    K = 6
    w = synth.World(pose=np.array([[*rng.uniform(-0.4, 0.4, 3), *_quat_axis_angle(rng.normal(size=3), 0.5)]
                                   for _ in range(K)]), half_ext=rng.uniform(0.05, 0.15, (K, 3)))
    lo, hi = np.asarray(rb.q_lo), np.asarray(rb.q_hi)
    u = rng.uniform(0.0, 1.0, (3, 7, rb.dof)) ** 0.25 * np.where(rng.uniform(size=(3, 7, rb.dof)) < 0.5, -1, 1)
    th = 0.5 * (lo + hi) + 0.45 * (hi - lo) * u
    qs = th[0, 0]
    goal = oracle_mod.goal_pose_from_fk(rb, th[0, -1])
    return rb, w, qs, goal, th


def test_state_outputs_brute_force(oracle_mod):
    """Per-state outputs of the evaluation against a recomputation from the
    pinned pieces (kinematics, sweep, self term, box distance): the world cost
    of state t is beta_2 sum_i v_i,t sum_k S_ik with the neighbours t - 1 and
    t + 1 of the padded sequence, the self cost beta_1 times the deepest pair,
    the clearance the smallest of every sphere-box and pair clearance; they add
    up to the trajectory's terms and decide its flag."""
    rb, w, qs, goal, th = _state_scene(oracle_mod)
    p = oracle_mod.params_default()
    out = oracle_mod.evaluate(rb, w, qs, goal, th, states=True)
    B, H, _ = th.shape
    M = len(rb.spheres)
    assert (out["state_terms"][:, :, 0] > 0).any() and (out["state_terms"][:, :, 1] > 0).any()
    for b in range(B):
        X = [oracle_mod.fk(rb, qs)[1]] + [oracle_mod.fk(rb, th[b, t])[1] for t in range(H)]
        for t in range(1, H + 1):
            tp = min(t + 1, H)
            world, clear = 0.0, np.inf
            for i in range(M):
                x0, x1, x2 = X[t - 1][i, :3], X[t][i, :3], X[tp][i, :3]
                r = X[t][i, 3]
                S = sum(oracle_mod.sweep_box(w.pose[k], w.half_ext[k], r, x0, x1, x2, p["eta"],
                                             p["sweep_steps"])[0] for k in range(len(w.pose)))
                v = np.linalg.norm(x2 - x0) / (2 * p["dt"])
                world += p["w_coll"] * v * S
                for k in range(len(w.pose)):
                    clear = min(clear, oracle_mod.box_sdf(w.pose[k], w.half_ext[k], x1)[0] - r)
            pen, _, _ = oracle_mod.self_penetration(rb, X[t])
            for i, j in rb.pairs:
                clear = min(clear, np.linalg.norm(X[t][i, :3] - X[t][j, :3]) - X[t][i, 3] - X[t][j, 3])
            assert out["state_terms"][b, t - 1, 0] == pytest.approx(world, rel=1e-12, abs=1e-12)
            assert out["state_terms"][b, t - 1, 1] == pytest.approx(p["w_self"] * pen, rel=1e-12, abs=1e-12)
            assert out["state_clear"][b, t - 1] == pytest.approx(clear, rel=1e-12, abs=1e-14)
    np.testing.assert_allclose(out["state_terms"].sum(1), out["terms"][:, :2], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(out["cfree"], (out["state_clear"] > 0).all(1))
    mg = np.minimum(out["state_margin"].min(1), np.abs(out["state_clear"]).min(1))
    np.testing.assert_allclose(out["margin"], mg, rtol=0, atol=0)


def test_state_margin_marks_self_argmax_tie(oracle_mod):
    """Two sphere pairs that penetrate equally at one state put that state's
    margin at zero (the gradient may go to either pair); the other states keep
    a margin away from zero.  Chain of three z joints one metre apart; folding
    joint 1 by pi brings link 2's frame back to the origin, turned by pi, so
    link 2's spheres (-0.625, 0) and (-0.625, -0.5) land 0.125 from link 0's
    spheres (0.5, 0) and (0.5, 0.5)."""
    ident = np.eye(3, 4).reshape(12)
    fixed = np.stack([ident] * 4)
    fixed[1, 3] = 1.0                              # F_1, F_2: one metre along x
    fixed[2, 3] = 1.0
    rb = synth.Robot(fixed_tf=fixed, axis=np.array([2, 2, 2], np.int32), q_lo=-4 * np.ones(3),
                     q_hi=4 * np.ones(3), v_max=np.ones(3), a_max=np.ones(3), j_max=np.ones(3),
                     spheres=np.array([[0.5, 0.0, 0, 0.1], [0.5, 0.5, 0, 0.1],
                                       [-0.625, 0.0, 0, 0.1], [-0.625, -0.5, 0, 0.1]]),
                     sphere_link=np.array([0, 0, 2, 2], np.int32), pairs=np.array([[0, 2], [1, 3]], np.int32))
    w = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    q_fold = np.array([0.0, math.pi, 0.0])
    _, sp, _ = oracle_mod.fk(rb, q_fold)
    d0 = np.linalg.norm(sp[0, :3] - sp[2, :3])
    d1 = np.linalg.norm(sp[1, :3] - sp[3, :3])
    assert d0 == pytest.approx(0.125, abs=1e-14) and d1 == pytest.approx(0.125, abs=1e-14)
    th = np.zeros((2, 3, 3))
    th[0, 1] = q_fold
    out = oracle_mod.evaluate(rb, w, np.zeros(3), np.array([0, 0, 1.0, 1, 0, 0, 0]), th,
                              dict(flags=oracle_mod.SELF | oracle_mod.SPEED | oracle_mod.SWEPT),
                              states=True)
    assert out["state_terms"][0, 1, 1] == pytest.approx(5000 * 0.075, rel=1e-12)
    assert out["state_margin"][0, 1] < 1e-12
    assert out["state_margin"][0, 0] > 0.1 and out["state_margin"][0, 2] > 0.1
    assert (out["state_margin"][1] > 0.1).all()
    # without the self term the tie decides nothing; the clearance still flags the contact
    out = oracle_mod.evaluate(rb, w, np.zeros(3), np.array([0, 0, 1.0, 1, 0, 0, 0]), th,
                              dict(flags=oracle_mod.SPEED | oracle_mod.SWEPT), states=True)
    assert (out["state_margin"] > 0.1).all()
    assert out["state_clear"][0, 1] == pytest.approx(-0.075, abs=1e-14) and not out["cfree"][0]


# ---------------------------------------------------------------------------
# Eq. 14 pose cost
# ---------------------------------------------------------------------------

def test_goal_cost_closed_forms(oracle_mod):
    p = oracle_mod.params_default()
    R = _rot(_quat_axis_angle([0.3, -1, 0.2], 0.8))
    ee = np.concatenate([R, np.array([[0.2], [0.1], [0.4]])], axis=1).reshape(12)
    q = oracle_mod._rot_to_quat(R)
    goal = np.array([0.2, 0.1, 0.4, *q])
    c, dp, dR = oracle_mod.goal_cost(p, ee, goal)
    assert c == pytest.approx(0.0, abs=1e-9)
    assert np.abs(dp).max() < 1e-9
    # quaternion sign does not matter
    c2, _, _ = oracle_mod.goal_cost(p, ee, np.array([0.2, 0.1, 0.4, *(-q)]))
    assert c2 == pytest.approx(c, abs=1e-12)
    # position error 1/alpha_2 along x: alpha_0 log cosh(1)
    goal_off = goal.copy()
    goal_off[0] += 1.0 / p["k_goal_pos"]
    c3, dp3, _ = oracle_mod.goal_cost(p, ee, goal_off)
    assert c3 == pytest.approx(p["w_goal_pos"] * math.log(math.cosh(1.0)), rel=1e-12)
    assert dp3[0] == pytest.approx(-p["w_goal_pos"] * p["k_goal_pos"] * math.tanh(1.0), rel=1e-12)
    # orientation error of angle phi about any axis: d_q = 1 - cos^2(phi/2) = sin^2(phi/2)
    phi = 0.3
    Rg = _rot(_quat_axis_angle([0, 0, 1], phi)) @ R
    qg = oracle_mod._rot_to_quat(Rg)
    c4, _, _ = oracle_mod.goal_cost(p, ee, np.array([0.2, 0.1, 0.4, *qg]))
    dq = math.sin(phi / 2) ** 2
    assert c4 == pytest.approx(p["w_goal_rot"] * math.log(math.cosh(p["k_goal_rot"] * dq)), rel=1e-10)


# ---------------------------------------------------------------------------
# whole evaluation: finite differences (sweep off; the sweep gradient is a
# surrogate by design, Sec. 3.4) and invariants
# ---------------------------------------------------------------------------

def _fd_problem(oracle_mod, n_joints, H, K, seed, flags_off=0):
    rb = _chain(n_joints, seed=seed)
    rng = np.random.default_rng(seed)
    w = synth.World(pose=np.array([[*rng.uniform(-0.2, 0.2, 3),
                                    *_quat_axis_angle(rng.normal(size=3), 0.7)]
                                   for _ in range(K)]).reshape(-1, 7),
                    half_ext=rng.uniform(0.1, 0.25, (K, 3)))
    qs = synth.uniform_config(rng, rb) * 0.6
    qg = synth.uniform_config(rng, rb) * 0.6
    goal = oracle_mod.goal_pose_from_fk(rb, qg)
    goal[:3] += 0.05
    th = synth.linear_seeds(rng, rb, qs, qg, 2, H, noise=0.2)
    return rb, w, qs, goal, th


def _fd_check(oracle_mod, rb, w, qs, goal, th, params, h=1e-6, rtol=2e-5):
    out = oracle_mod.evaluate(rb, w, qs, goal, th, params)
    g = out["grad"]
    num = np.zeros_like(th)
    it = np.nditer(th, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        cp = oracle_mod.evaluate(rb, w, qs, goal, tp, params, want_grad=False)["cost"][idx[0]]
        cm = oracle_mod.evaluate(rb, w, qs, goal, tm, params, want_grad=False)["cost"][idx[0]]
        num[idx] = (cp - cm) / (2 * h)
    for b in range(th.shape[0]):
        err = np.linalg.norm(num[b] - g[b])
        assert err <= rtol * np.linalg.norm(num[b]) + 1e-6, (b, err, np.linalg.norm(num[b]))
    return out


@pytest.mark.parametrize("n_joints,H", [(2, 5), (3, 6), (7, 6)])
def test_gradient_finite_difference_trajopt(oracle_mod, n_joints, H):
    rb, w, qs, goal, th = _fd_problem(oracle_mod, n_joints, H, 3, seed=n_joints)
    p = dict(flags=oracle_mod.SPEED | oracle_mod.SELF, dt=0.1)
    out = _fd_check(oracle_mod, rb, w, qs, goal, th, p)
    assert (out["terms"][:, 0] > 0).any(), "the world term must be active for this pin"


def test_gradient_finite_difference_each_term(oracle_mod):
    """FD per term: switch all other weights off, so a dropped term cannot
    hide behind a large one."""
    rb, w, qs, goal, th = _fd_problem(oracle_mod, 7, 6, 3, seed=21)
    base = dict(flags=oracle_mod.SPEED | oracle_mod.SELF | oracle_mod.VEL_COST, dt=0.1)
    zero = dict(w_goal_pos=0.0, w_goal_rot=0.0, w_coll=0.0, w_self=0.0, w_bound=0.0,
                w_acc=0.0, w_jerk=0.0, w_vel=0.0)
    for keys in [("w_coll",), ("w_self",), ("w_goal_pos",), ("w_goal_rot",), ("w_bound",),
                 ("w_acc",), ("w_jerk",), ("w_vel",)]:
        p = dict(base, **zero)
        for k in keys:
            p[k] = oracle_mod.params_default()[k]
        _fd_check(oracle_mod, rb, w, qs, goal, th, p)


def test_gradient_finite_difference_ik(oracle_mod):
    rb, w, qs, goal, th = _fd_problem(oracle_mod, 7, 1, 4, seed=9)
    p = dict(flags=oracle_mod.IK_MODE | oracle_mod.SELF)
    th = np.random.default_rng(2).uniform(rb.q_lo, rb.q_hi, (3, 1, rb.dof)) * 0.5
    _fd_check(oracle_mod, rb, w, qs, goal, th, p)


def test_terms_sum_and_stationary_sphere_has_no_world_cost(oracle_mod):
    """Eq. 11 scales by the sphere speed: a trajectory that holds the start
    state inside a box costs nothing in the world term, but is not free."""
    rb = _robot()
    q = np.zeros(rb.dof)
    _, sp, _ = oracle_mod.fk(rb, q)
    w = synth.World(pose=np.array([[*sp[10, :3], 1, 0, 0, 0]]), half_ext=np.full((1, 3), 0.1))
    th = np.tile(q, (1, 5, 1))
    out = oracle_mod.evaluate(rb, w, q, np.array([0, 0, 1.0, 1, 0, 0, 0]), th)
    assert out["terms"][0, 0] == 0.0
    assert not out["cfree"][0]
    assert out["cost"][0] == pytest.approx(out["terms"][0].sum(), rel=1e-15)
    # moving through the same box costs
    th2 = th.copy()
    th2[0, 2:, 0] += 0.3
    out2 = oracle_mod.evaluate(rb, w, q, np.array([0, 0, 1.0, 1, 0, 0, 0]), th2)
    assert out2["terms"][0, 0] > 0


def test_free_flag_against_brute_force(oracle_mod):
    rb = _robot()
    rng = np.random.default_rng(8)
    qs = synth.uniform_config(rng, rb)
    w = synth.make_world(6, 2)
    th = synth.linear_seeds(rng, rb, qs, synth.uniform_config(rng, rb), 6, 8)
    out = oracle_mod.evaluate(rb, w, qs, np.array([0, 0, 1.0, 1, 0, 0, 0]), th)
    for b in range(6):
        free = True
        for t in range(8):
            _, sp, _ = oracle_mod.fk(rb, th[b, t])
            for i in range(rb.n_spheres):
                for k in range(w.n):
                    phi, _ = oracle_mod.box_sdf(w.pose[k], w.half_ext[k], sp[i, :3])
                    free &= phi - sp[i, 3] > 0
            for i, j in rb.pairs:
                free &= np.linalg.norm(sp[i, :3] - sp[j, :3]) - sp[i, 3] - sp[j, 3] > 0
        assert bool(out["cfree"][b]) == bool(free)


# ---------------------------------------------------------------------------
# L-BFGS two-loop (App. A.7) and line search (Alg. 1)
# ---------------------------------------------------------------------------

def _dense_bfgs_direction(S, Y, g):
    """Explicit BFGS inverse-Hessian recursion H+ = (I - rho s y^T) H (I - rho y s^T) + rho s s^T
    from H0 = gamma I, over the valid pairs oldest to newest."""
    n = g.size
    valid = [(s, y) for s, y in zip(S, Y) if y @ s > 1e-8]
    if not valid:
        return -g
    s_new, y_new = valid[-1]
    H = (s_new @ y_new) / (y_new @ y_new) * np.eye(n)
    for s, y in valid:
        rho = 1.0 / (y @ s)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return -H @ g


def test_two_loop_equals_dense_bfgs(oracle_mod):
    rng = np.random.default_rng(0)
    n, m = 12, 6
    A = rng.normal(size=(n, n))
    A = A @ A.T + n * np.eye(n)
    st = oracle_mod.LbfgsState(n, m)
    x = rng.normal(size=n)
    S, Y = [], []
    for k in range(9):
        st.x[:] = x
        st.g[:] = A @ x + 0.1 * np.sin(x)        # mildly non-quadratic
        d = st.direction()
        if k > 0:
            S.append(x - xp)
            Y.append(st.g - gp)
        ref = _dense_bfgs_direction(S[-m:], Y[-m:], st.g)
        np.testing.assert_allclose(d, ref, rtol=1e-10, atol=1e-12)
        assert d @ st.g < 0                        # descent
        xp, gp = x.copy(), st.g.copy()
        x = x + 0.3 * d


def test_two_loop_secant_condition(oracle_mod):
    """BFGS keeps H y = s for the newest pair: feeding g = y_newest gives d = -s."""
    rng = np.random.default_rng(1)
    n, m = 8, 4
    A = np.diag(rng.uniform(1, 5, n))
    st = oracle_mod.LbfgsState(n, m)
    x = rng.normal(size=n)
    for k in range(5):
        st.x[:] = x
        st.g[:] = A @ x
        d = st.direction()
        x = x + 0.5 * d
    # one more update with the new point, then probe with g := y_newest
    st.x[:] = x
    st.g[:] = A @ x
    st.direction()
    s_new, y_new = st.s[-1].copy(), st.y[-1].copy()
    probe = oracle_mod.LbfgsState(n, m)
    probe.s[:], probe.y[:], probe.rho[:] = st.s, st.y, st.rho
    probe.g[:] = y_new
    probe.iter[0] = 0                                 # no further history update
    d = probe.direction()
    np.testing.assert_allclose(d, -s_new, rtol=1e-10, atol=1e-12)


def test_two_loop_first_step_and_inert_pair(oracle_mod):
    n, m = 5, 3
    st = oracle_mod.LbfgsState(n, m)
    st.g[:] = np.arange(1, 6.0)
    np.testing.assert_allclose(st.direction(), -st.g)     # no history: steepest descent
    # a step with y^T s <= 1e-8 leaves an inert pair: direction is still -g
    st.x[:] += 1e-6
    d = st.direction()
    assert st.rho[-1] == 0.0
    np.testing.assert_allclose(d, -st.g)


def test_line_search_on_quadratic(oracle_mod):
    """f(x) = a/2 x^2 from x0 with d = -f'(x0): candidate alpha gives
    f = f0 (1 - a alpha)^2.  Armijo with c1 holds iff (1-a alpha)^2 <= 1 - 2 c1 a alpha;
    weak Wolfe with c2 holds iff (1 - a alpha) <= c2."""
    a, x0 = 2.0, 1.5
    f = lambda x: 0.5 * a * x * x
    g0 = np.array([a * x0])
    d = -g0
    p = dict(alpha=[0.01, 0.1, 0.3, 0.5, 0.9, 1.0], armijo_c1=1e-4, wolfe_c2=0.9)
    xs = x0 + np.array(p["alpha"]) * d[0]
    cc = f(xs)
    cg = (a * xs)[:, None]
    for wolfe in (False, True):
        flags = oracle_mod.WOLFE if wolfe else 0
        idx, _ = oracle_mod.ls_select(dict(p, flags=flags), f(x0), g0, d, cc, cg)
        exp = 0
        for l, al in enumerate(p["alpha"]):
            ok = (1 - a * al) ** 2 <= 1 - 2 * 1e-4 * a * al
            if wolfe:
                ok = ok and (1 - a * al) <= 0.9
            if ok:
                exp = l
        assert idx == exp
    # no candidate passes: fall back to index 0 (the 0.01 step)
    idx, _ = oracle_mod.ls_select(dict(p, flags=0), f(x0), g0, d, cc + 100.0, cg)
    assert idx == 0


def test_candidates_are_clipped(oracle_mod):
    p = dict(alpha=[0.5, 2.0])
    x = np.array([0.0, 0.9, -0.9, 0.0])
    d = np.array([1.0, 1.0, -1.0, -1.0])
    cand = oracle_mod.ls_candidates(p, x, d, [-1.0, -2.0], [1.0, 2.0], 2)
    np.testing.assert_allclose(cand[0], [0.5, 1.4, -1.0, -0.5])
    np.testing.assert_allclose(cand[1], [1.0, 2.0, -1.0, -2.0])


def test_solve_best_cost_never_increases(oracle_mod):
    rb = _robot()
    rng = np.random.default_rng(2)
    qs = synth.uniform_config(rng, rb)
    w = synth.make_world(3, 9, lambda p, h: oracle_mod.start_collides_with_box(rb, qs, p, h))
    pr = synth.make_problem(rb, w, 3, 2, 8, lambda q: oracle_mod.goal_pose_from_fk(rb, q), qs)
    init = oracle_mod.evaluate(rb, w, qs, pr.goal, pr.seeds)["cost"]
    prev = init
    for iters in (1, 3, 6):
        out = oracle_mod.solve(rb, w, qs, pr.goal, pr.seeds, iters)
        assert np.all(out["cost"] <= prev + 1e-9)
        prev = out["cost"]
        ev = oracle_mod.evaluate(rb, w, qs, pr.goal, out["x"])
        np.testing.assert_allclose(ev["cost"], out["cost"], rtol=1e-12)
    assert np.all(prev < init)


# ---------------------------------------------------------------------------
# Sec. 4.2 particle-based optimisation (Eq. 12, Eq. 13)
# ---------------------------------------------------------------------------

def test_particle_sample_closed_forms(oracle_mod):
    mu = np.array([0.5, -1.0, 2.0])
    sigma = np.array([4.0, 0.25, 0.0])
    eps = np.array([[0.0, 0.0, 0.0], [1.0, -2.0, 3.0]])
    p = oracle_mod.particle_sample(mu, sigma, eps)
    assert np.array_equal(p[0], mu)                       # zero noise: the mean
    assert np.allclose(p[1], [0.5 + 2.0, -1.0 - 1.0, 2.0])  # sqrt(sigma) scales the noise


def test_particle_equal_costs_reduce_to_plain_averages(oracle_mod):
    rng = np.random.default_rng(0)
    n, n_p = 5, 7
    th = rng.normal(size=(n_p, n))
    mu, sigma = rng.normal(size=n), rng.uniform(0.1, 1.0, size=n)
    k_mu, k_s = 0.3, 0.6
    m2, s2, w = oracle_mod.particle_update(np.full(n_p, 3.25), th, mu, sigma, 0.7, k_mu, k_s)
    assert np.allclose(w, 1.0 / n_p)
    assert np.allclose(m2, (1 - k_mu) * mu + k_mu * th.mean(axis=0), atol=1e-14)
    assert np.allclose(s2, (1 - k_s) * sigma + k_s * ((th - mu) ** 2).mean(axis=0), atol=1e-14)


def test_particle_weights_follow_exponential_utility(oracle_mod):
    th = np.array([[0.0], [1.0]])
    beta = 2.5
    _, _, w = oracle_mod.particle_update(np.array([10.0, 13.0]), th, [0.0], [1.0], beta, 1.0, 1.0)
    assert np.isclose(w.sum(), 1.0) and np.all(w > 0)
    assert np.isclose(w[1] / w[0], np.exp(-(13.0 - 10.0) / beta))   # c = -C / beta
    # a common shift of every cost changes nothing
    _, _, w2 = oracle_mod.particle_update(np.array([1e6 + 10.0, 1e6 + 13.0]), th, [0.0], [1.0], beta,
                                          1.0, 1.0)
    assert np.allclose(w2, w, rtol=1e-12)


def test_particle_temperature_limits(oracle_mod):
    rng = np.random.default_rng(1)
    n, n_p = 4, 6
    th = rng.normal(size=(n_p, n))
    cost = rng.uniform(0.0, 10.0, size=n_p)
    mu, sigma = np.zeros(n), np.ones(n)
    best = int(np.argmin(cost))
    # beta -> 0: all weight on the cheapest particle
    m2, s2, w = oracle_mod.particle_update(cost, th, mu, sigma, 1e-9, 1.0, 1.0)
    assert np.isclose(w[best], 1.0) and np.allclose(m2, th[best]) and np.allclose(s2, th[best] ** 2)
    # beta -> infinity: uniform weights
    _, _, w = oracle_mod.particle_update(cost, th, mu, sigma, 1e12, 1.0, 1.0)
    assert np.allclose(w, 1.0 / n_p)


def test_particle_rates_zero_keep_state_and_one_particle_replaces_it(oracle_mod):
    mu, sigma = np.array([0.2, -0.4]), np.array([0.3, 0.5])
    th = np.array([[1.0, 2.0]])
    m2, s2, _ = oracle_mod.particle_update([7.0], th, mu, sigma, 1.0, 0.0, 0.0)
    assert np.array_equal(m2, mu) and np.array_equal(s2, sigma)
    m2, s2, _ = oracle_mod.particle_update([7.0], th, mu, sigma, 1.0, 1.0, 1.0)
    assert np.allclose(m2, th[0]) and np.allclose(s2, (th[0] - mu) ** 2)   # deviation from the old mean


def test_particle_covariance_recovers_sampling_variance(oracle_mod):
    """Equal costs, k = 1: the new covariance is the weighted second moment of
    the particles about the old mean, which for mu + sqrt(sigma) * N(0, 1)
    samples converges to sigma."""
    rng = np.random.default_rng(2)
    mu, sigma = np.array([0.3, -0.7, 1.1]), np.array([0.04, 0.25, 1.0])
    eps = rng.standard_normal((200000, 3))
    th = oracle_mod.particle_sample(mu, sigma, eps)
    m2, s2, _ = oracle_mod.particle_update(np.zeros(len(th)), th, mu, sigma, 1.0, 1.0, 1.0)
    assert np.allclose(s2, sigma, rtol=0.02)
    assert np.allclose(m2, mu, atol=0.01)


# ---------------------------------------------------------------------------
# Eq. 15 joint-space goal cost (App. A.1)
# ---------------------------------------------------------------------------

def test_cspace_goal_closed_form_and_zero_at_goal(oracle_mod):
    """One trajectory whose last state differs from the goal configuration in
    one joint by d: the goal term grows by alpha_4 logcosh(alpha_5 d^2); at the
    goal it adds nothing, value or gradient."""
    from paper_2310_17274_gb300 import synth
    rb = synth.make_robot(synth.SPHERES_42, seed=0)
    w = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    H = 4
    rng = np.random.default_rng(3)
    th = rng.uniform(-0.5, 0.5, size=(1, H, rb.dof))
    q0 = th[0, 0].copy()
    goal7 = np.array([0.3, 0.0, 0.4, 1.0, 0.0, 0.0, 0.0])
    base = oracle_mod.evaluate(rb, w, q0, goal7, th)
    p = dict(flags=oracle_mod.params_default()["flags"] | oracle_mod.CSPACE_GOAL)
    at = oracle_mod.evaluate(rb, w, q0, goal7, th, p, goal_q=th[0, -1])
    assert at["terms"][0, 4] == base["terms"][0, 4]
    assert np.array_equal(at["grad"], base["grad"])
    d = 0.07
    gq = th[0, -1].copy()
    gq[2] += d
    off = oracle_mod.evaluate(rb, w, q0, goal7, th, p, goal_q=gq)
    expect = 5000.0 * np.log(np.cosh(50.0 * d * d))
    assert off["terms"][0, 4] - base["terms"][0, 4] == pytest.approx(expect, rel=1e-12)
    # its gradient only touches theta_H, along the offset joint, pulling toward the goal
    dg = off["grad"] - base["grad"]
    assert np.all(dg[0, :-1] == 0.0)
    assert dg[0, -1, 2] == pytest.approx(-2.0 * 5000.0 * 50.0 * np.tanh(50.0 * d * d) * d, rel=1e-9)
    assert np.count_nonzero(dg[0, -1]) == 1


def test_cspace_goal_gradient_finite_differences(oracle_mod):
    from paper_2310_17274_gb300 import synth
    rb = synth.make_robot(synth.SPHERES_42, seed=0)
    w = synth.make_world(4, 1)
    H = 6
    rng = np.random.default_rng(4)
    th = rng.uniform(-0.6, 0.6, size=(1, H, rb.dof))
    q0 = rng.uniform(-0.6, 0.6, size=rb.dof)
    gq = rng.uniform(-0.6, 0.6, size=rb.dof)
    goal7 = np.array([0.3, 0.1, 0.4, 1.0, 0.0, 0.0, 0.0])
    p = dict(flags=oracle_mod.params_default()["flags"] | oracle_mod.CSPACE_GOAL)
    ref = oracle_mod.evaluate(rb, w, q0, goal7, th, p, goal_q=gq)
    h = 1e-6
    for j in range(rb.dof):
        tp, tm = th.copy(), th.copy()
        tp[0, -1, j] += h
        tm[0, -1, j] -= h
        fd = (oracle_mod.evaluate(rb, w, q0, goal7, tp, p, goal_q=gq)["cost"][0] -
              oracle_mod.evaluate(rb, w, q0, goal7, tm, p, goal_q=gq)["cost"][0]) / (2 * h)
        assert fd == pytest.approx(ref["grad"][0, -1, j], rel=2e-5, abs=1e-4)


# ---------------------------------------------------------------------------
# Sec. 5 Alg. "Parallel Steering"
# ---------------------------------------------------------------------------

def test_steer_steps_closed_form(oracle_mod):
    edges = np.zeros((3, 2, 7))
    edges[0, 1, 2] = 0.95
    edges[1, 1, 4] = -0.31
    edges[2, 0, 6] = 0.5
    assert oracle_mod.steer_steps(edges, 0.1) == 10          # floor(9.5) + 1
    assert oracle_mod.steer_steps(edges[1:2], 0.1) == 4       # floor(3.1) + 1


def _first_invalid_brute_force(oracle_mod, rb, w, a, b, n):
    """Per-sample clearance from the kinematics and the box distance alone."""
    for i in range(n + 1):
        q = a + (i / n) * (b - a)
        _, sp, _ = oracle_mod.fk(rb, q)
        for k in range(w.n):
            for s in range(len(sp)):
                if sp[s, 3] < 0:
                    continue
                if not (oracle_mod.box_sdf(w.pose[k], w.half_ext[k], sp[s, :3])[0] - sp[s, 3] > 0):
                    return i
        for (i1, j1) in rb.pairs:
            if np.linalg.norm(sp[i1, :3] - sp[j1, :3]) - sp[i1, 3] - sp[j1, 3] <= 0:
                return i
    return n + 1


def test_steer_free_edge_and_box_on_the_way(oracle_mod):
    from paper_2310_17274_gb300 import synth
    rb = synth.make_robot(synth.SPHERES_42, seed=0)
    a = np.array([0.0, 0.3, 0.0, -0.4, 0.0, 0.2, 0.0])
    b = np.array([1.2, -0.2, 0.5, 0.3, -0.6, 0.9, 0.4])
    edges = np.stack([a, b])[None]
    n = oracle_mod.steer_steps(edges, 0.05)
    empty = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    assert _first_invalid_brute_force(oracle_mod, rb, empty, a, b, n) == n + 1, "self-colliding edge"
    last, v, d = oracle_mod.steer(rb, empty, edges, n)
    assert last[0] == n and np.allclose(v[0], b) and d[0] == pytest.approx(np.linalg.norm(b - a))
    # a small box centred on the end effector's sphere at 60 % of the way
    i_star = int(0.6 * n)
    _, sp, _ = oracle_mod.fk(rb, a + (i_star / n) * (b - a))
    s = int(np.argmax(np.where(rb.sphere_link == rb.dof - 1, 1, 0)))
    w = synth.World(pose=np.array([[*sp[s, :3], 1.0, 0.0, 0.0, 0.0]]), half_ext=np.full((1, 3), 0.02))
    first = _first_invalid_brute_force(oracle_mod, rb, w, a, b, n)
    assert 0 < first <= i_star
    last, v, d = oracle_mod.steer(rb, w, edges, n)
    assert last[0] == first - 1
    assert np.allclose(v[0], a + (last[0] / n) * (b - a))
    assert d[0] == pytest.approx(np.linalg.norm(v[0] - a))


def test_steer_start_in_collision(oracle_mod):
    from paper_2310_17274_gb300 import synth
    rb = synth.make_robot(synth.SPHERES_42, seed=0)
    a = np.zeros(7)
    b = np.full(7, 0.3)
    _, sp, _ = oracle_mod.fk(rb, a)
    w = synth.World(pose=np.array([[*sp[10, :3], 1.0, 0.0, 0.0, 0.0]]), half_ext=np.full((1, 3), 0.05))
    last, v, d = oracle_mod.steer(rb, w, np.stack([a, b])[None], 5)
    assert last[0] == -1 and np.array_equal(v[0], a) and d[0] == 0.0


# ---------------------------------------------------------------------------
# App. "Time-step Discretization": retime
# ---------------------------------------------------------------------------

def test_retime_scaling_and_limits(oracle_mod):
    """A trajectory retimed to dt is at the limit at dt: the largest of the
    velocity, acceleration and jerk ratios (App. A.5 stencils at dt) is 1; a
    constant trajectory needs no time at all."""
    from paper_2310_17274_gb300 import synth
    rb = synth.make_robot(synth.SPHERES_42, seed=0)
    H = 20
    rng = np.random.default_rng(6)
    q0 = rng.uniform(-0.3, 0.3, size=rb.dof)
    th = q0 + np.cumsum(rng.normal(0, 0.05, size=(H, rb.dof)), axis=0)
    dt = oracle_mod.retime(rb, q0, th)
    v, a, j = oracle_mod.stencil(q0, th, dt)
    ratio = max(np.max(np.abs(v) / rb.v_max), np.max(np.abs(a) / rb.a_max), np.max(np.abs(j) / rb.j_max))
    assert ratio == pytest.approx(1.0, rel=1e-12)
    # the same shape twice as large in every joint: each ratio grows by 2,
    # so dt grows by 2, sqrt(2) or cbrt(2) depending on the binding limit
    dt2 = oracle_mod.retime(rb, q0, q0 + 2.0 * (th - q0))
    assert dt2 / dt == pytest.approx(2.0) or dt2 / dt == pytest.approx(np.sqrt(2.0)) or \
        dt2 / dt == pytest.approx(np.cbrt(2.0))
    assert oracle_mod.retime(rb, q0, np.tile(q0, (H, 1))) < 1e-6   # rounding residue only (cube root)


def test_time_scaled_weights_keep_smoothness(oracle_mod):
    """Reading of Alg. "Time Discretization"'s weight scaling: with the weight
    on the square of the k-th derivative times (dt / dt0)^(2k), the Eq. 16
    smoothness of the same waypoints is the same at every dt (the App. A.5
    derivatives scale as 1/dt^k); without the jerk term only the
    acceleration part is left."""
    rb = _robot()
    rng = np.random.default_rng(40)
    qs = synth.uniform_config(rng, rb) * 0.3
    th = synth.linear_seeds(rng, rb, qs, synth.uniform_config(rng, rb) * 0.3, 3, 12, noise=0.3)
    w = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    goal = np.array([0, 0, 1.0, 1, 0, 0, 0])
    base = dict(flags=oracle_mod.SPEED | oracle_mod.SWEPT, w_jerk=2.0)
    ref = oracle_mod.evaluate(rb, w, qs, goal, th, base)["terms"][:, 3]
    for dt in (0.01, 0.02, 0.25, 0.7):
        p = oracle_mod.time_scaled_params(base, dt)
        r = dt / 0.05
        assert p["dt"] == dt and p["w_acc"] == pytest.approx(5000 * r ** 4, rel=1e-14)
        assert p["w_jerk"] == pytest.approx(2.0 * r ** 6, rel=1e-14)
        assert p["w_vel"] == pytest.approx(5000 * r ** 2, rel=1e-14)
        got = oracle_mod.evaluate(rb, w, qs, goal, th, p)["terms"][:, 3]
        np.testing.assert_allclose(got, ref, rtol=1e-9)
        acc_only = oracle_mod.evaluate(rb, w, qs, goal, th, dict(base, w_jerk=0.0))["terms"][:, 3]
        got = oracle_mod.evaluate(rb, w, qs, goal, th, oracle_mod.time_scaled_params(base, dt, jerk=False))
        np.testing.assert_allclose(got["terms"][:, 3], acc_only, rtol=1e-9)


def test_time_discretized_solve_stages(oracle_mod):
    """Alg. "Time Discretization" as composed: the first solve is the plain
    solve at the coarse step without jerk; dt_opt is the retimed step of its
    best seed; the second solve starts from its seeds with the weights for
    dt_opt; every seed is retimed, and the chosen one has the lowest score
    among the collision-free seeds, which puts it exactly at a limit."""
    rb = _robot()
    rng = np.random.default_rng(41)
    qs = synth.uniform_config(rng, rb) * 0.5
    qg = synth.uniform_config(rng, rb) * 0.5
    w = synth.make_world(3, 7, lambda p, h: oracle_mod.start_collides_with_box(rb, qs, p, h))
    goal = oracle_mod.goal_pose_from_fk(rb, qg)
    seeds = synth.linear_seeds(rng, rb, qs, qg, 4, 12, noise=0.2)
    out = oracle_mod.time_discretized_solve(rb, w, qs, goal, seeds, 6, 6)
    p1 = oracle_mod.time_scaled_params(None, 0.25, jerk=False)
    s1 = oracle_mod.solve(rb, w, qs, goal, seeds, 6, p1)
    c1, f1 = s1["cost"], s1["cfree"]
    b1 = int(np.argmin(np.where(f1, c1, np.inf))) if f1.any() else int(np.argmin(c1))
    np.testing.assert_array_equal(out["first"], s1["x"][b1])
    dt_opt = max(oracle_mod.retime(rb, qs, s1["x"][b1]), 1e-3)
    assert out["stage"][4] == dt_opt
    p2 = oracle_mod.time_scaled_params(None, dt_opt, jerk=True)
    np.testing.assert_array_equal(out["stage"], [p1["dt"], p1["w_vel"], p1["w_acc"], p1["w_jerk"],
                                                 p2["dt"], p2["w_vel"], p2["w_acc"], p2["w_jerk"]])
    assert p1["w_jerk"] == 0.0 and p2["w_jerk"] > 0.0
    s2 = oracle_mod.solve(rb, w, qs, goal, s1["x"], 6, p2)
    np.testing.assert_array_equal(out["traj"], s2["x"])
    for b in range(4):
        assert out["dt"][b] == oracle_mod.retime(rb, qs, out["traj"][b])
    ok = np.where(out["cfree"], out["score"], np.inf)
    if out["cfree"].any():
        assert out["chosen"] == int(np.argmin(ok))
        x = out["traj"][out["chosen"]]
        v, a, j = oracle_mod.stencil(qs, x, out["dt"][out["chosen"]])
        ratio = max(np.max(np.abs(v) / rb.v_max), np.max(np.abs(a) / rb.a_max), np.max(np.abs(j) / rb.j_max))
        assert ratio == pytest.approx(1.0, rel=1e-9)
    else:
        assert out["chosen"] == int(np.argmin(out["cost"]))


def _axis_angle(axis, phi):
    """Rotation matrix about a unit axis (Rodrigues), for the pose-error pins."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(phi) * K + (1 - math.cos(phi)) * K @ K


def _quat(R):
    """wxyz of a rotation matrix (Shepperd's method, trace branch + fallbacks)."""
    tr = np.trace(R)
    if tr > 0:
        s = math.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    else:
        i = int(np.argmax(np.diag(R)))
        j, k = (i + 1) % 3, (i + 2) % 3
        s = math.sqrt(1.0 + R[i, i] - R[j, j] - R[k, k]) * 2
        q = [0.0] * 4
        q[0] = (R[k, j] - R[j, k]) / s
        q[1 + i] = 0.25 * s
        q[1 + j] = (R[j, i] + R[i, j]) / s
        q[1 + k] = (R[k, i] + R[i, k]) / s
    q = np.asarray(q)
    return q / np.linalg.norm(q)


def test_pose_error_closed_forms(oracle_mod):
    """App. "Solver details" pose error |p - p_g| + d_q: a goal displaced by a
    vector delta with the same orientation gives |delta|; a goal rotated by
    phi about any axis through the end effector gives (1 - cos phi) / 2."""
    rb = synth.make_robot(synth.SPHERES_42, seed=0)
    rng = np.random.default_rng(40)
    q = synth.uniform_config(rng, rb)
    _, _, ee = oracle_mod.fk(rb, q)
    E = np.asarray(ee).reshape(3, 4)
    p, R = E[:, 3], E[:, :3]
    delta = np.array([0.03, -0.04, 0.12])
    assert oracle_mod.pose_error(rb, q, np.concatenate([p + delta, _quat(R)])) == \
        pytest.approx(np.linalg.norm(delta), abs=1e-12)
    for phi in (0.1, 1.0, 2.5):
        Rg = R @ _axis_angle(rng.normal(size=3), phi)
        assert oracle_mod.pose_error(rb, q, np.concatenate([p, _quat(Rg)])) == \
            pytest.approx((1 - math.cos(phi)) / 2, abs=1e-12)


def test_rank_seeds_closed_forms_and_choice(oracle_mod):
    """Seed scores of App. "Solver details": at rest on the goal only the motion
    time H dt remains; IK at the goal configuration scores w_dist |q - q0|; the
    largest jerk equals a direct evaluation of the five-point stencil on the
    padded sequence; the choice is the lowest collision-free score, the lowest
    index on ties, never a NaN score, -1 without a collision-free seed."""
    rb = synth.make_robot(synth.SPHERES_42, seed=0)
    rng = np.random.default_rng(41)
    D, H = rb.dof, 16
    q0 = synth.uniform_config(rng, rb)
    qg = synth.uniform_config(rng, rb)
    goal = oracle_mod.goal_pose_from_fk(rb, qg)
    rest = np.tile(qg, (1, H, 1))
    s, b = oracle_mod.rank_seeds(rb, qg, goal, rest, [1], dt_all=0.04, w_pose=1.0, w_jerk=1e-3, w_time=2.0)
    assert s[0] == pytest.approx(2.0 * H * 0.04, abs=1e-9) and b == 0
    s, _ = oracle_mod.rank_seeds(rb, q0, goal, qg[None, None, :], [1], ik=True, w_pose=1.0, w_dist=0.3)
    assert s[0] == pytest.approx(0.3 * np.linalg.norm(qg - q0), abs=1e-9)
    # largest jerk by brute force: ext = [q0 q0 q0 theta_1..theta_H theta_H theta_H]
    th = q0 + np.cumsum(rng.normal(0, 0.05, size=(3, H, D)), axis=1)
    dts = np.array([0.03, 0.05, 0.08])
    s, _ = oracle_mod.rank_seeds(rb, q0, goal, th, [1, 1, 1], dt=dts, w_pose=0.0, w_jerk=1.0, w_time=0.0)
    for k in range(3):
        ext = np.concatenate([np.tile(q0, (3, 1)), th[k], np.tile(th[k][-1], (2, 1))])
        jm = max(abs(-ext[e - 2, j] + 2 * ext[e - 1, j] - 2 * ext[e + 1, j] + ext[e + 2, j]) / (2 * dts[k] ** 3)
                 for e in range(2, H + 3) for j in range(D))
        assert s[k] == pytest.approx(jm, rel=1e-12)
    # choice: seeds 1 and 3 tie and are the lowest collision-free; seed 0 lower but not free;
    # seed 2 NaN
    th4 = np.stack([rest[0], rest[0], rest[0], rest[0]])
    th4[2, -1, 0] = np.nan   # the last state: its pose error is NaN
    s, b = oracle_mod.rank_seeds(rb, qg, goal, th4, [0, 1, 1, 1], dt=np.array([0.01, 0.02, 0.01, 0.02]),
                                 w_pose=1.0, w_jerk=0.0, w_time=1.0)
    assert np.isnan(s[2]) and b == 1
    _, b = oracle_mod.rank_seeds(rb, qg, goal, th4, [0, 0, 0, 0], dt_all=0.05)
    assert b == -1


def test_ik_without_self_check(oracle_mod):
    """IK without collision checking (Sec. 6): with the self term off and the
    no-self-check flag, a configuration folded onto itself is reported free
    when no box is near, and its cost is unchanged; without the flag the same
    configuration is not free."""
    rb = synth.make_robot(synth.SPHERES_60, seed=0)
    rng = np.random.default_rng(42)
    lo, hi = np.asarray(rb.q_lo), np.asarray(rb.q_hi)
    world = synth.World(pose=np.zeros((0, 7)), half_ext=np.zeros((0, 3)))
    goal = oracle_mod.goal_pose_from_fk(rb, synth.uniform_config(rng, rb))
    q0 = synth.uniform_config(rng, rb)
    found = None
    for _ in range(200):
        u = rng.uniform(0.0, 1.0, rb.dof) ** 0.25 * np.where(rng.uniform(size=rb.dof) < 0.5, -1, 1)
        q = 0.5 * (lo + hi) + 0.5 * (hi - lo) * u
        _, sph, _ = oracle_mod.fk(rb, q)
        pen, _, _ = oracle_mod.self_penetration(rb, sph)
        if pen > 1e-3:
            found = q
            break
    assert found is not None
    th = found[None, None, :]
    plain = oracle_mod.evaluate(rb, world, q0, goal, th, dict(flags=oracle_mod.IK_MODE))
    nocheck = oracle_mod.evaluate(rb, world, q0, goal, th,
                                  dict(flags=oracle_mod.IK_MODE | oracle_mod.NO_SELF_CHECK))
    assert not plain["cfree"][0] and nocheck["cfree"][0]
    assert nocheck["cost"][0] == plain["cost"][0]
