"""FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

A plain, slow, single-threaded C99 implementation (``cro.c``) of what the hot
path computes, written from the paper's equations (arXiv 2310.17274, Sec. 3-4
and App. A).  It shares no code with the CUDA library.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may load
it; the library never does.

Every input is a plain array (float64 unless stated); robot / world objects
are read by attribute (``fixed_tf``, ``axis``, ``q_lo`` ... as produced by
``paper_2310_17274_gb300.synth``), so this module imports nothing from the
library package.

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
against closed forms, invariants, brute force or finite differences; the
end-to-end optimised trajectories (many chaotic iterations) are "parity
unpinned" and only checked distributionally.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cro.c")
_LIB_PATH = os.path.join(_HERE, "libcro.so")
_lock = threading.Lock()
_lib = None

SWEPT, SPEED, SELF, WOLFE, STRONG_WOLFE, IK_MODE, VEL_COST, CSPACE_GOAL = 1, 2, 4, 8, 16, 32, 64, 128
NO_SELF_CHECK = 256
N_TERMS = 5
MAX_ALPHA = 16

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint8)


class _Robot(C.Structure):
    _fields_ = [("dof", C.c_int32), ("fixed_tf", _dp), ("axis", _ip), ("q_lo", _dp),
                ("q_hi", _dp), ("v_max", _dp), ("a_max", _dp), ("j_max", _dp),
                ("n_spheres", C.c_int32), ("spheres", _dp), ("sphere_link", _ip),
                ("n_pairs", C.c_int32), ("pairs", _ip)]


class _World(C.Structure):
    _fields_ = [("n", C.c_int32), ("pose", _dp), ("half_ext", _dp)]


class _Params(C.Structure):
    _fields_ = [("w_goal_pos", C.c_double), ("w_goal_rot", C.c_double),
                ("k_goal_pos", C.c_double), ("k_goal_rot", C.c_double),
                ("w_coll", C.c_double), ("w_self", C.c_double), ("w_bound", C.c_double),
                ("w_acc", C.c_double), ("w_jerk", C.c_double), ("w_vel", C.c_double),
                ("k_vel", C.c_double), ("eta", C.c_double), ("eta_bound", C.c_double),
                ("dt", C.c_double), ("sweep_steps", C.c_int32), ("history", C.c_int32),
                ("n_alpha", C.c_int32), ("alpha", C.c_double * MAX_ALPHA),
                ("armijo_c1", C.c_double), ("wolfe_c2", C.c_double), ("flags", C.c_uint32),
                ("w_cspace", C.c_double), ("k_cspace", C.c_double)]


class _Lbfgs(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("x", _dp), ("g", _dp), ("c", _dp),
                ("x_prev", _dp), ("g_prev", _dp), ("s", _dp), ("y", _dp), ("rho", _dp),
                ("iter", _ip)]


def build(force: bool = False) -> str:
    """Compile cro.c into oracle/libcro.so with the host gcc (plain -O2, no
    fast-math, no target-specific flags, so x86 and Arm give the same results)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or \
                os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(os.path.join(_HERE, "cro.h"))):
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                                   "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        L.cro_params_default.argtypes = [C.POINTER(_Params)]
        L.cro_fk.argtypes = [C.POINTER(_Robot), _dp, _dp, _dp, _dp]
        L.cro_box_sdf.argtypes = [_dp, _dp, _dp, _dp]
        L.cro_box_sdf.restype = C.c_double
        L.cro_smooth_distance.argtypes = [C.c_double, C.c_double, _dp]
        L.cro_smooth_distance.restype = C.c_double
        L.cro_bound_cost.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        L.cro_bound_cost.restype = C.c_double
        L.cro_sweep_box.argtypes = [_dp, _dp, C.c_double, _dp, _dp, _dp, C.c_double, C.c_int32,
                                    _dp, _dp]
        L.cro_sweep_box.restype = C.c_double
        L.cro_self_penetration.argtypes = [C.POINTER(_Robot), _dp, _ip, _dp]
        L.cro_self_penetration.restype = C.c_double
        L.cro_stencil.argtypes = [C.c_int32, C.c_int32, _dp, _dp, C.c_double, _dp, _dp, _dp]
        L.cro_goal_cost.argtypes = [C.POINTER(_Params), _dp, _dp, _dp, _dp]
        L.cro_goal_cost.restype = C.c_double
        L.cro_eval.argtypes = [C.POINTER(_Robot), C.POINTER(_World), _dp, _dp, _dp,
                               C.POINTER(_Params), C.c_int32, _dp, C.c_int32, _dp, _dp, _up,
                               _dp, _dp]
        L.cro_eval_states.argtypes = [C.POINTER(_Robot), C.POINTER(_World), _dp, _dp, _dp,
                                      C.POINTER(_Params), C.c_int32, _dp, C.c_int32, _dp, _dp, _up,
                                      _dp, _dp, _dp, _dp, _dp]
        L.cro_time_scaled_params.argtypes = [C.POINTER(_Params), C.c_double, C.c_int32, C.POINTER(_Params)]
        L.cro_time_discretized_solve.argtypes = [C.POINTER(_Robot), C.POINTER(_World), _dp, _dp, _dp,
                                                 C.POINTER(_Params), C.c_int32, C.c_int32, _dp, C.c_int32,
                                                 C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double,
                                                 C.c_double, _dp, _dp, _dp, _dp, _up, _dp, _dp]
        L.cro_time_discretized_solve.restype = C.c_int32
        L.cro_lbfgs_direction.argtypes = [C.POINTER(_Lbfgs), _dp]
        L.cro_ls_candidates.argtypes = [C.POINTER(_Params), C.c_int32, C.c_int32, _dp, _dp,
                                        _dp, _dp, _dp]
        L.cro_retime.argtypes = [C.POINTER(_Robot), C.c_int32, _dp, _dp]
        L.cro_retime.restype = C.c_double
        L.cro_pose_error.argtypes = [C.POINTER(_Robot), _dp, _dp]
        L.cro_pose_error.restype = C.c_double
        L.cro_rank_seeds.argtypes = [C.POINTER(_Robot), C.c_int32, C.c_int32, _dp, _dp, _dp,
                                     C.POINTER(C.c_uint8), _dp, C.c_double, C.c_int32, C.c_double,
                                     C.c_double, C.c_double, C.c_double, _dp]
        L.cro_rank_seeds.restype = C.c_int32
        L.cro_steer_steps.argtypes = [C.c_int32, C.c_int32, _dp, C.c_double]
        L.cro_steer_steps.restype = C.c_int32
        L.cro_steer.argtypes = [C.POINTER(_Robot), C.POINTER(_World), C.c_int32, _dp, C.c_int32, _ip,
                                _dp, _dp]
        L.cro_particle_sample.argtypes = [C.c_int32, C.c_int32, _dp, _dp, _dp, _dp]
        L.cro_particle_update.argtypes = [C.c_int32, C.c_int32, _dp, _dp, C.c_double, C.c_double,
                                          C.c_double, _dp, _dp, _dp]
        L.cro_ls_select.argtypes = [C.POINTER(_Params), C.c_int32, C.c_double, _dp, _dp, _dp,
                                    _dp, _dp]
        L.cro_ls_select.restype = C.c_int32
        L.cro_solve.argtypes = [C.POINTER(_Robot), C.POINTER(_World), _dp, _dp, _dp,
                                C.POINTER(_Params), C.c_int32, C.c_int32, _dp, C.c_int32, _dp,
                                _dp, _up]
        _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t=_dp):
    if a is None:
        return None
    return a.ctypes.data_as(t)


class _Keep:
    """Holds the numpy arrays a ctypes struct points into."""

    def __init__(self):
        self.refs = []

    def __call__(self, a):
        self.refs.append(a)
        return a


def _robot(rb, keep):
    s = _Robot()
    s.dof = int(len(rb.axis))
    s.fixed_tf = _p(keep(_f64(rb.fixed_tf)))
    s.axis = _p(keep(_i32(rb.axis)), _ip)
    s.q_lo = _p(keep(_f64(rb.q_lo)))
    s.q_hi = _p(keep(_f64(rb.q_hi)))
    s.v_max = _p(keep(_f64(rb.v_max)))
    s.a_max = _p(keep(_f64(rb.a_max)))
    s.j_max = _p(keep(_f64(rb.j_max)))
    s.n_spheres = int(len(rb.spheres))
    s.spheres = _p(keep(_f64(rb.spheres)))
    s.sphere_link = _p(keep(_i32(rb.sphere_link)), _ip)
    s.n_pairs = int(len(rb.pairs))
    s.pairs = _p(keep(_i32(np.asarray(rb.pairs).reshape(-1, 2))), _ip)
    return s


def _world(w, keep):
    s = _World()
    pose = keep(_f64(np.asarray(w.pose).reshape(-1, 7)))
    he = keep(_f64(np.asarray(w.half_ext).reshape(-1, 3)))
    s.n = int(len(pose))
    s.pose = _p(pose)
    s.half_ext = _p(he)
    return s


def params_default() -> dict:
    p = _Params()
    lib().cro_params_default(C.byref(p))
    return _params_to_dict(p)


def _params_to_dict(p):
    d = {}
    for name, _ in _Params._fields_:
        v = getattr(p, name)
        if name == "alpha":
            v = [float(x) for x in v][: p.n_alpha]
        d[name] = v
    return d


def _params(d=None):
    base = params_default()
    if d:
        base.update(d)
    p = _Params()
    for name, _ in _Params._fields_:
        if name == "alpha":
            al = list(base["alpha"])
            if len(al) > MAX_ALPHA:
                raise ValueError("too many step sizes")
            for i, a in enumerate(al):
                p.alpha[i] = float(a)
            p.n_alpha = len(al)
        elif name == "n_alpha":
            continue
        else:
            setattr(p, name, base[name])
    return p


# ---------------------------------------------------------------------------
# pieces
# ---------------------------------------------------------------------------

def fk(rb, theta):
    """Forward kinematics of one configuration -> (link_tf [dof,12], spheres [M,4], ee [12])."""
    keep = _Keep()
    R = _robot(rb, keep)
    dof, M = R.dof, R.n_spheres
    th = _f64(theta)
    lt = np.zeros((dof, 12))
    sp = np.zeros((M, 4))
    ee = np.zeros(12)
    lib().cro_fk(C.byref(R), _p(th), _p(lt), _p(sp), _p(ee))
    return lt, sp, ee


def box_sdf(pose7, half_ext, x):
    g = np.zeros(3)
    phi = lib().cro_box_sdf(_p(_f64(pose7)), _p(_f64(half_ext)), _p(_f64(x)), _p(g))
    return phi, g


def smooth_distance(d, eta):
    s = C.c_double()
    v = lib().cro_smooth_distance(float(d), float(eta), C.byref(s))
    return v, s.value


def bound_cost(q, lo, hi, eta2):
    s = C.c_double()
    v = lib().cro_bound_cost(float(q), float(lo), float(hi), float(eta2), C.byref(s))
    return v, s.value


def sweep_box(pose7, half_ext, r, x0, x1, x2, eta, steps):
    g = np.zeros(3)
    m = C.c_double(np.finfo(np.float64).max)
    x0a = None if x0 is None else _f64(x0)
    x2a = None if x2 is None else _f64(x2)
    S = lib().cro_sweep_box(_p(_f64(pose7)), _p(_f64(half_ext)), float(r), _p(x0a),
                            _p(_f64(x1)), _p(x2a), float(eta), int(steps), _p(g), C.byref(m))
    return S, g, m.value


def self_penetration(rb, spheres_world):
    keep = _Keep()
    R = _robot(rb, keep)
    X = _f64(spheres_world)
    arg = C.c_int32()
    g = np.zeros((R.n_spheres, 3))
    pen = lib().cro_self_penetration(C.byref(R), _p(X), C.byref(arg), _p(g))
    return pen, arg.value, g


def stencil(q0, theta, dt):
    th = _f64(theta)
    H, dof = th.shape
    v = np.zeros((H + 1, dof))
    a = np.zeros((H + 1, dof))
    j = np.zeros((H + 1, dof))
    lib().cro_stencil(H, dof, _p(_f64(q0)), _p(th), float(dt), _p(v), _p(a), _p(j))
    return v, a, j


def goal_cost(params, ee, goal7):
    P = _params(params)
    dp = np.zeros(3)
    dR = np.zeros(9)
    c = lib().cro_goal_cost(C.byref(P), _p(_f64(ee)), _p(_f64(goal7)), _p(dp), _p(dR))
    return c, dp, dR.reshape(3, 3)


# ---------------------------------------------------------------------------
# whole evaluation and optimiser
# ---------------------------------------------------------------------------

def evaluate(rb, world, q_start, goal7, theta, params=None, want_grad=True, goal_q=None, states=False):
    """Cost, gradient, collision-free flag, per-term costs and decision margin
    of trajectories theta [B,H,dof] (one problem).  With states=True also the
    per-state outputs of cro_eval_states: state_terms [B,H,2] (world, self
    cost of each state), state_margin [B,H] (distance of the state's cost- and
    gradient-setting decisions from their thresholds) and state_clear [B,H]
    (the state's smallest clearance; collision-free when > 0)."""
    keep = _Keep()
    R = _robot(rb, keep)
    W = _world(world, keep)
    P = _params(params)
    th = _f64(theta)
    B, H, dof = th.shape
    cost = np.zeros(B)
    grad = np.zeros((B, H, dof)) if want_grad else None
    cfree = np.zeros(B, dtype=np.uint8)
    terms = np.zeros((B, N_TERMS))
    margin = np.zeros(B)
    gq = None if goal_q is None else _f64(goal_q)
    if not states:
        lib().cro_eval(C.byref(R), C.byref(W), _p(_f64(q_start)), _p(_f64(goal7)), _p(gq), C.byref(P),
                       H, _p(th), B, _p(cost), _p(grad), _p(cfree, _up), _p(terms), _p(margin))
        return dict(cost=cost, grad=grad, cfree=cfree.astype(bool), terms=terms, margin=margin)
    st_terms = np.zeros((B, H, 2))
    st_margin = np.zeros((B, H))
    st_clear = np.zeros((B, H))
    lib().cro_eval_states(C.byref(R), C.byref(W), _p(_f64(q_start)), _p(_f64(goal7)), _p(gq),
                          C.byref(P), H, _p(th), B, _p(cost), _p(grad), _p(cfree, _up), _p(terms),
                          _p(margin), _p(st_terms), _p(st_margin), _p(st_clear))
    return dict(cost=cost, grad=grad, cfree=cfree.astype(bool), terms=terms, margin=margin,
                state_terms=st_terms, state_margin=st_margin, state_clear=st_clear)


class LbfgsState:
    """One seed's optimiser state, in the oracle's own layout (newest pair last)."""

    def __init__(self, n, m):
        self.n, self.m = n, m
        self.x = np.zeros(n)
        self.g = np.zeros(n)
        self.c = np.zeros(1)
        self.x_prev = np.zeros(n)
        self.g_prev = np.zeros(n)
        self.s = np.zeros((m, n))
        self.y = np.zeros((m, n))
        self.rho = np.zeros(m)
        self.iter = np.zeros(1, dtype=np.int32)

    def direction(self):
        st = _Lbfgs(self.n, self.m, _p(self.x), _p(self.g), _p(self.c), _p(self.x_prev),
                    _p(self.g_prev), _p(self.s), _p(self.y), _p(self.rho), _p(self.iter, _ip))
        d = np.zeros(self.n)
        lib().cro_lbfgs_direction(C.byref(st), _p(d))
        return d


def ls_candidates(params, x, d, q_lo, q_hi, dof):
    P = _params(params)
    x = _f64(x)
    n = x.size
    cand = np.zeros((P.n_alpha, n))
    lib().cro_ls_candidates(C.byref(P), n, dof, _p(_f64(q_lo)), _p(_f64(q_hi)), _p(x),
                            _p(_f64(d)), _p(cand))
    return cand


def ls_select(params, c0, g0, d, cand_cost, cand_grad):
    P = _params(params)
    g0 = _f64(g0)
    n = g0.size
    m = C.c_double()
    idx = lib().cro_ls_select(C.byref(P), n, float(c0), _p(g0), _p(_f64(d)),
                              _p(_f64(cand_cost)), _p(_f64(np.asarray(cand_grad).reshape(-1, n))),
                              C.byref(m))
    return idx, m.value


def solve(rb, world, q_start, goal7, seeds, iters, params=None, goal_q=None):
    keep = _Keep()
    R = _robot(rb, keep)
    W = _world(world, keep)
    P = _params(params)
    sd = _f64(seeds)
    B, H, dof = sd.shape
    bx = np.zeros_like(sd)
    bc = np.zeros(B)
    bf = np.zeros(B, dtype=np.uint8)
    gq = None if goal_q is None else _f64(goal_q)
    lib().cro_solve(C.byref(R), C.byref(W), _p(_f64(q_start)), _p(_f64(goal7)), _p(gq), C.byref(P), H,
                    B, _p(sd), int(iters), _p(bx), _p(bc), _p(bf, _up))
    return dict(x=bx, cost=bc, cfree=bf.astype(bool))


def goal_pose_from_fk(rb, q):
    """Goal pose (xyz + quaternion wxyz) reached by configuration q, via the
    oracle's own FK.  Used by tests to make reachable goals."""
    _, _, ee = fk(rb, q)
    R = ee.reshape(3, 4)[:, :3]
    return np.concatenate([ee.reshape(3, 4)[:, 3], _rot_to_quat(R)])


def _rot_to_quat(R):
    # Shepperd's method (largest-pivot branch), result with w >= 0
    tr = np.trace(R)
    if tr > 0:
        s = np.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    q /= np.linalg.norm(q)
    return q if q[0] >= 0 else -q


def start_collides_with_box(rb, q_start, pose7, half_ext):
    """True when the start configuration's spheres touch the box (discrete
    clearance <= 0).  Used by tests as the world generator's rejection test."""
    _, sp, _ = fk(rb, q_start)
    for i in range(len(sp)):
        if sp[i, 3] < 0:
            continue
        phi, _ = box_sdf(pose7, half_ext, sp[i, :3])
        if phi - sp[i, 3] <= 0:
            return True
    return False


# ---------------------------------------------------------------------------
# Sec. 4.2 particle-based optimisation
# ---------------------------------------------------------------------------

def particle_sample(mu, sigma, eps):
    """particles [n_p, n] = mu + sqrt(sigma) * eps (eps [n_p, n])."""
    mu, sigma, eps = _f64(mu), _f64(sigma), _f64(eps)
    n = mu.size
    n_p = eps.size // n
    out = np.zeros((n_p, n))
    lib().cro_particle_sample(n, n_p, _p(mu), _p(sigma), _p(eps), _p(out))
    return out


def particle_update(cost, particles, mu, sigma, beta, k_mu, k_sigma):
    """One UPDATE of the particle optimiser; returns (mu, sigma, weights)."""
    cost, particles = _f64(cost), _f64(particles)
    mu, sigma = _f64(mu).copy(), _f64(sigma).copy()
    n, n_p = mu.size, cost.size
    w = np.zeros(n_p)
    lib().cro_particle_update(n, n_p, _p(cost), _p(particles), float(beta), float(k_mu),
                              float(k_sigma), _p(mu), _p(sigma), _p(w))
    return mu, sigma, w


# ---------------------------------------------------------------------------
# Sec. 5 parallel steering
# ---------------------------------------------------------------------------

def steer_steps(edges, r):
    """n of Alg. "Parallel Steering" for edges [E, 2, dof] at resolution r."""
    e = _f64(edges)
    return int(lib().cro_steer_steps(e.shape[0], e.shape[2], _p(e), float(r)))


def steer(rb, world, edges, n):
    """Last valid sample index, last valid configuration and its distance per edge."""
    keep = _Keep()
    R = _robot(rb, keep)
    W = _world(world, keep)
    e = _f64(edges)
    E, _, dof = e.shape
    last = np.zeros(E, dtype=np.int32)
    v = np.zeros((E, dof))
    d = np.zeros(E)
    lib().cro_steer(C.byref(R), C.byref(W), E, _p(e), int(n), _p(last, _ip), _p(v), _p(d))
    return last, v, d


# ---------------------------------------------------------------------------
# App. "Time-step Discretization"
# ---------------------------------------------------------------------------

def pose_error(rb, q, goal7):
    """|p - p_g| + d_q of the end effector at configuration q (App. "Solver details")."""
    keep = _Keep()
    R = _robot(rb, keep)
    return float(lib().cro_pose_error(C.byref(R), _p(_f64(q)), _p(_f64(goal7))))


def rank_seeds(rb, q0, goal7, theta, cfree, dt=None, dt_all=None, ik=False, w_pose=1.0, w_jerk=1e-3,
               w_time=1.0, w_dist=0.1):
    """Scores of seeds theta [B,H,dof] and the index of the lowest-scoring
    collision-free one (-1 when none), App. "Solver details"."""
    keep = _Keep()
    R = _robot(rb, keep)
    th = _f64(theta)
    B, H, dof = th.shape
    score = np.zeros(B)
    cf = np.ascontiguousarray(np.asarray(cfree, dtype=np.uint8))
    dtp = None if dt is None else _f64(dt)
    best = lib().cro_rank_seeds(C.byref(R), H, B, _p(_f64(q0)), _p(_f64(goal7)), _p(th),
                                cf.ctypes.data_as(C.POINTER(C.c_uint8)), _p(dtp),
                                float(0.0 if dt_all is None else dt_all), int(bool(ik)), float(w_pose),
                                float(w_jerk), float(w_time), float(w_dist), _p(score))
    return score, int(best)


def retime(rb, q0, theta):
    """dt that puts one trajectory theta [H, dof] at the robot's limits."""
    keep = _Keep()
    R = _robot(rb, keep)
    th = _f64(theta)
    return float(lib().cro_retime(C.byref(R), th.shape[0], _p(_f64(q0)), _p(th)))


def time_scaled_params(params, dt, jerk=True) -> dict:
    """cro_time_scaled_params: the parameters for step dt (weights on the k-th
    derivative's square times (dt / dt0)^(2k); jerk=False zeroes the jerk weight)."""
    P = _params(params)
    out = _Params()
    lib().cro_time_scaled_params(C.byref(P), float(dt), int(bool(jerk)), C.byref(out))
    return _params_to_dict(out)


def time_discretized_solve(rb, world, q_start, goal7, seeds, iters1, iters2, params=None, dt_init=0.25,
                           dt_min=1e-3, w_pose=1.0, w_jerk=1e-3, w_time=1.0, goal_q=None):
    """Alg. "Time Discretization" (cro_time_discretized_solve) for one problem."""
    keep = _Keep()
    R = _robot(rb, keep)
    W = _world(world, keep)
    P = _params(params)
    sd = _f64(seeds)
    B, H, dof = sd.shape
    first = np.zeros((H, dof))
    stage = np.zeros(8)
    traj = np.zeros_like(sd)
    cost = np.zeros(B)
    cfree = np.zeros(B, dtype=np.uint8)
    dt = np.zeros(B)
    score = np.zeros(B)
    gq = None if goal_q is None else _f64(goal_q)
    chosen = lib().cro_time_discretized_solve(
        C.byref(R), C.byref(W), _p(_f64(q_start)), _p(_f64(goal7)), _p(gq), C.byref(P), H, B, _p(sd),
        int(iters1), int(iters2), float(dt_init), float(dt_min), float(w_pose), float(w_jerk), float(w_time),
        _p(first), _p(stage), _p(traj), _p(cost), _p(cfree, _up), _p(dt), _p(score))
    return dict(first=first, stage=stage, traj=traj, cost=cost, cfree=cfree.astype(bool), dt=dt, score=score,
                chosen=int(chosen))
