"""Thin ctypes binding of libcrgb.so (include/crgb.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch provides device memory and the current stream.  There
is no CPU fallback: loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrgb.so")
_lock = threading.Lock()
_lib = None

SWEPT, SPEED, SELF, WOLFE, STRONG_WOLFE, IK_MODE, VEL_COST, CSPACE_GOAL = 1, 2, 4, 8, 16, 32, 64, 128
NO_SELF_CHECK = 256
N_TERMS = 5
MAX_ALPHA = 16

_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)
_up = C.POINTER(C.c_uint8)
_vp = C.c_void_p


class CrError(RuntimeError):
    """A failed call; `status` is its cr_status code."""

    def __init__(self, msg, status=1):
        super().__init__(msg)
        self.status = status


class RobotDesc(C.Structure):
    _fields_ = [("dof", C.c_int32), ("fixed_tf", _fp), ("axis", _ip), ("q_lo", _fp),
                ("q_hi", _fp), ("v_max", _fp), ("a_max", _fp), ("j_max", _fp),
                ("n_spheres", C.c_int32), ("spheres", _fp), ("sphere_link", _ip),
                ("n_pairs", C.c_int32), ("pairs", _ip)]


class WorldDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("pose", _fp), ("half_ext", _fp)]


class Params(C.Structure):
    _fields_ = [("w_goal_pos", C.c_float), ("w_goal_rot", C.c_float),
                ("k_goal_pos", C.c_float), ("k_goal_rot", C.c_float),
                ("w_coll", C.c_float), ("w_self", C.c_float), ("w_bound", C.c_float),
                ("w_acc", C.c_float), ("w_jerk", C.c_float), ("w_vel", C.c_float),
                ("k_vel", C.c_float), ("eta", C.c_float), ("eta_bound", C.c_float),
                ("dt", C.c_float), ("sweep_steps", C.c_int32), ("history", C.c_int32),
                ("n_alpha", C.c_int32), ("alpha", C.c_float * MAX_ALPHA),
                ("armijo_c1", C.c_float), ("wolfe_c2", C.c_float), ("flags", C.c_uint32),
                ("w_cspace", C.c_float), ("k_cspace", C.c_float)]


class Problem(C.Structure):
    _fields_ = [("world", _vp), ("q_start", _fp), ("goal", _fp), ("n_seeds", C.c_int32),
                ("horizon", C.c_int32), ("seeds", _fp), ("goal_q", _fp)]


class Result(C.Structure):
    _fields_ = [("traj", _vp), ("cost", _vp), ("cfree", _vp), ("best", _vp), ("status", _vp)]


class ParticleConfig(C.Structure):
    _fields_ = [("iters", C.c_int32), ("n_particles", C.c_int32), ("beta", C.c_float), ("k_mu", C.c_float),
                ("k_sigma", C.c_float), ("sigma0", C.c_float), ("eps", _vp)]


class TimeoptConfig(C.Structure):
    _fields_ = [("dt_init", C.c_float), ("dt_min", C.c_float), ("iters1", C.c_int32),
                ("iters2", C.c_int32), ("w_pose", C.c_float), ("w_jerk", C.c_float), ("w_time", C.c_float)]


class TimeoptResult(C.Structure):
    _fields_ = [("first", _vp), ("stage", _vp), ("dt", _vp), ("score", _vp), ("chosen", _vp)]


SOLVE_GRAPH, SOLVE_PERSISTENT, SOLVE_DEVICE_SEEDS = 1, 2, 4


class OptState(C.Structure):
    _fields_ = [("n_seeds", C.c_int32), ("horizon", C.c_int32),
                ("x", _vp), ("g", _vp), ("c", _vp), ("x_prev", _vp), ("g_prev", _vp),
                ("s", _vp), ("y", _vp), ("rho", _vp), ("iter", _vp), ("dir", _vp),
                ("cand", _vp), ("cand_cost", _vp), ("cand_grad", _vp), ("cand_cfree", _vp),
                ("best_x", _vp), ("best_c", _vp), ("best_cfree", _vp), ("ls_index", _vp)]


# name -> (argtypes, restype); the exported symbols of include/crgb.h
SIGNATURES = {
    "cr_last_error": ([], C.c_char_p),
    "cr_version": ([], C.c_char_p),
    "cr_params_default": ([C.POINTER(Params)], None),
    "cr_measure_ffma": ([C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_float), _vp], C.c_int32),
    "cr_robot_create": ([C.POINTER(RobotDesc), C.POINTER(_vp)], C.c_int32),
    "cr_robot_destroy": ([_vp], None),
    "cr_world_create": ([C.POINTER(WorldDesc), C.POINTER(_vp)], C.c_int32),
    "cr_world_destroy": ([_vp], None),
    "cr_fk": ([_vp, _vp, C.c_int32, _vp, _vp, _vp, _vp], C.c_int32),
    "cr_eval": ([_vp, C.POINTER(Problem), C.POINTER(Params), _vp, C.c_int32, _vp, _vp, _vp, _vp,
                 _vp, _vp], C.c_int32),
    "cr_opt_propose": ([_vp, C.POINTER(Params), C.POINTER(OptState), _vp], C.c_int32),
    "cr_opt_select": ([_vp, C.POINTER(Params), C.POINTER(OptState), _vp], C.c_int32),
    "cr_context_create": ([C.c_int, C.c_size_t, C.POINTER(_vp)], C.c_int32),
    "cr_context_destroy": ([_vp], None),
    "cr_solve": ([_vp, _vp, C.c_int32, C.POINTER(Problem), C.POINTER(Params), C.c_int32, C.c_uint32,
                  C.POINTER(Result), _vp], C.c_int32),
    "cr_particle_step": ([_vp, C.POINTER(Problem), C.POINTER(Params), C.c_int32, C.c_int32, _vp,
                          _vp, _vp, _vp, _vp, C.c_float, C.c_float, C.c_float, _vp], C.c_int32),
    "cr_steer": ([_vp, _vp, C.c_int32, _vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp], C.c_int32),
    "cr_retime": ([_vp, C.POINTER(Problem), C.c_int32, _vp, _vp, _vp], C.c_int32),
    "cr_rank_seeds": ([_vp, C.POINTER(Problem), C.POINTER(Params), C.c_int32, _vp, _vp, _vp, C.c_float,
                       C.c_float, C.c_float, C.c_float, _vp, _vp, _vp], C.c_int32),
    "cr_solve_particles": ([_vp, _vp, C.c_int32, C.POINTER(Problem), C.POINTER(Params), C.c_int32, C.c_uint32,
                            C.POINTER(ParticleConfig), C.POINTER(Result), _vp], C.c_int32),
    "cr_solve_timeopt": ([_vp, _vp, C.c_int32, C.POINTER(Problem), C.POINTER(Params),
                          C.POINTER(TimeoptConfig), C.c_uint32, C.POINTER(Result), C.POINTER(TimeoptResult),
                          _vp], C.c_int32),
    "cr_autotune": ([_vp, _vp, C.c_int32, C.POINTER(Problem), C.POINTER(Params), C.c_int32,
                     C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                     C.POINTER(C.c_float)], C.c_int32),
    "cr_tune_set": ([_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32],
                    C.c_int32),
    "cr_server_create": ([_vp, _vp, _vp, C.POINTER(_vp)], C.c_int32),
    "cr_server_destroy": ([_vp], None),
    "cr_server_submit": ([_vp, C.c_int32, C.POINTER(Problem), C.POINTER(C.c_uint64)], C.c_int32),
    "cr_server_step": ([_vp, _vp], C.c_int32),
    "cr_server_poll": ([_vp, C.c_uint64, C.POINTER(C.c_int32), _vp, _vp, _vp, C.POINTER(C.c_int32),
                        C.POINTER(C.c_int32)], C.c_int32),
    "cr_server_wait": ([_vp, C.c_uint64, C.c_int32], C.c_int32),
    "cr_server_snapshot": ([_vp, C.c_uint64, _vp, C.POINTER(C.c_size_t)], C.c_int32),
    "cr_server_restore": ([_vp, _vp, C.c_size_t, _vp, C.POINTER(C.c_uint64)], C.c_int32),
    "cr_server_stats": ([_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_size_t)],
                        C.c_int32),
    "cr_eval_batch_noalloc": ([_vp, C.c_int32, C.POINTER(Problem), C.POINTER(Params), _ip, _vp, _vp,
                               _vp, _vp, _vp, _vp], C.c_int32),
}


def lib():
    """Load libcrgb.so; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise CrError(f"{LIB_PATH} is missing: build it first "
                                  "(python -m paper_2310_17274_gb300.build)")
                L = C.CDLL(LIB_PATH)
                for name, (argt, rest) in SIGNATURES.items():
                    fn = getattr(L, name)
                    fn.argtypes = argt
                    fn.restype = rest
                _lib = L
    return _lib


def check(status: int, what: str = "") -> None:
    if status != 0:
        msg = lib().cr_last_error().decode()
        raise CrError(f"{what} failed with status {status}: {msg}", status)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, t=_fp):
    return None if a is None else a.ctypes.data_as(t)


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise CrError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# handles
# ---------------------------------------------------------------------------

class Robot:
    """Device copy of a robot description (fields as in synth.Robot)."""

    def __init__(self, rb):
        self.dof = int(len(rb.axis))
        self.n_spheres = int(len(rb.spheres))
        self.n_pairs = int(len(rb.pairs))
        keep = [_f32(rb.fixed_tf), _i32(rb.axis), _f32(rb.q_lo), _f32(rb.q_hi), _f32(rb.v_max),
                _f32(rb.a_max), _f32(rb.j_max), _f32(rb.spheres), _i32(rb.sphere_link),
                _i32(np.asarray(rb.pairs).reshape(-1, 2))]
        d = RobotDesc(self.dof, _p(keep[0]), _p(keep[1], _ip), _p(keep[2]), _p(keep[3]),
                      _p(keep[4]), _p(keep[5]), _p(keep[6]), self.n_spheres, _p(keep[7]),
                      _p(keep[8], _ip), self.n_pairs, _p(keep[9], _ip))
        h = _vp()
        check(lib().cr_robot_create(C.byref(d), C.byref(h)), "cr_robot_create")
        self.handle = h
        self.q_lo = np.asarray(rb.q_lo, dtype=np.float64)
        self.q_hi = np.asarray(rb.q_hi, dtype=np.float64)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.cr_robot_destroy(h)
            self.handle = None


class World:
    def __init__(self, w):
        pose = _f32(np.asarray(w.pose).reshape(-1, 7))
        he = _f32(np.asarray(w.half_ext).reshape(-1, 3))
        self.n = int(len(pose))
        d = WorldDesc(self.n, _p(pose), _p(he))
        h = _vp()
        check(lib().cr_world_create(C.byref(d), C.byref(h)), "cr_world_create")
        self.handle = h

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.cr_world_destroy(h)
            self.handle = None


def params_default() -> dict:
    p = Params()
    lib().cr_params_default(C.byref(p))
    d = {}
    for name, _ in Params._fields_:
        v = getattr(p, name)
        if name == "alpha":
            v = [float(x) for x in v][: p.n_alpha]
        d[name] = v
    return d


def make_params(over: dict | None = None) -> Params:
    base = params_default()
    if over:
        base.update(over)
    p = Params()
    for name, _ in Params._fields_:
        if name == "alpha":
            al = list(base["alpha"])
            if len(al) > MAX_ALPHA:
                raise CrError("too many step sizes")
            for i, a in enumerate(al):
                p.alpha[i] = float(a)
            p.n_alpha = len(al)
        elif name == "n_alpha":
            continue
        else:
            setattr(p, name, base[name])
    return p


class ProblemSpec:
    """Host-side arrays of one problem, kept alive for the ctypes struct."""

    def __init__(self, world: World, q_start, goal, horizon: int, seeds=None, goal_q=None):
        self.world = world
        self.q_start = _f32(q_start)
        self.goal = _f32(goal)
        self.horizon = int(horizon)
        self.seeds = None if seeds is None else _f32(seeds)
        self.goal_q = None if goal_q is None else _f32(goal_q)
        self._struct = None

    def struct(self) -> Problem:
        """The ctypes view of this problem, built once (the arrays it points
        to live as long as this object)."""
        if self._struct is None:
            B = 0 if self.seeds is None else int(self.seeds.shape[0])
            self._struct = Problem(self.world.handle, _p(self.q_start), _p(self.goal), B, self.horizon,
                                   _p(self.seeds), _p(self.goal_q))
        return self._struct


# ---------------------------------------------------------------------------
# hot-path calls
# ---------------------------------------------------------------------------

def measure_ffma(iters=400000, stream=None):
    """FP32 FMA throughput of the current device (cr_measure_ffma): (TFLOP/s, ms)."""
    t, ms = C.c_float(), C.c_float()
    check(lib().cr_measure_ffma(int(iters), C.byref(t), C.byref(ms), _stream(stream)), "cr_measure_ffma")
    return t.value, ms.value


def fk(robot: Robot, theta, spheres=True, ee=True, link_tf=False, stream=None):
    """Forward kinematics of theta (CUDA tensor [N, dof])."""
    import torch
    theta = theta.contiguous()
    n = theta.shape[0]
    dev = theta.device
    sp = torch.empty((n, robot.n_spheres, 4), device=dev) if spheres else None
    e = torch.empty((n, 12), device=dev) if ee else None
    lt = torch.empty((n, robot.dof, 12), device=dev) if link_tf else None
    check(lib().cr_fk(robot.handle, _dptr(theta), n, _dptr(sp), _dptr(e), _dptr(lt),
                      _stream(stream)), "cr_fk")
    return sp, e, lt


def evaluate(robot: Robot, problem: ProblemSpec, theta, params=None, want_grad=True,
             want_terms=True, want_states=False, stream=None):
    """Cost, gradient, collision-free flags and per-term costs of theta
    (CUDA float32 tensor [B, H, dof]) in one fused launch; with want_states
    also the world and self cost of every state ([B, H, 2])."""
    import torch
    theta = theta.contiguous()
    B = theta.shape[0]
    dev = theta.device
    cost = torch.empty(B, device=dev)
    grad = torch.empty_like(theta) if want_grad else None
    cfree = torch.empty(B, device=dev, dtype=torch.uint8)
    terms = torch.empty((B, N_TERMS), device=dev) if want_terms else None
    states = torch.empty((B, theta.shape[1], 2), device=dev) if want_states else None
    P = params if isinstance(params, Params) else make_params(params)
    pr = problem.struct()
    check(lib().cr_eval(robot.handle, C.byref(pr), C.byref(P), _dptr(theta), B, _dptr(cost),
                        _dptr(grad), _dptr(cfree), _dptr(terms), _dptr(states), _stream(stream)),
          "cr_eval")
    return dict(cost=cost, grad=grad, cfree=cfree, terms=terms, state_terms=states)


def particle_step(robot: Robot, problem: ProblemSpec, mu, sigma, eps, params=None, beta=1.0,
                  k_mu=0.9, k_sigma=0.9, particles=None, cost=None, stream=None):
    """One particle-optimisation iteration (cr_particle_step) for the seeds of
    one problem.  mu, sigma: CUDA float32 [B, H, dof], updated in place; eps:
    [B, n_particles, H, dof] unit Gaussian samples.  Returns (particles, cost)."""
    import torch
    B, n_p = eps.shape[0], eps.shape[1]
    if particles is None:
        particles = torch.empty_like(eps)
    if cost is None:
        cost = torch.empty((B, n_p), device=eps.device)
    P = params if isinstance(params, Params) else make_params(params)
    pr = problem.struct()
    for t in (mu, sigma, eps, particles, cost):
        if not t.is_contiguous():
            raise ValueError("particle_step: tensors must be contiguous")
    check(lib().cr_particle_step(robot.handle, C.byref(pr), C.byref(P), int(B), int(n_p), _dptr(mu),
                                 _dptr(sigma), _dptr(eps), _dptr(particles), _dptr(cost),
                                 float(beta), float(k_mu), float(k_sigma), _stream(stream)),
          "cr_particle_step")
    return particles, cost


def steer_steps(edges, r):
    """n of the parallel-steering algorithm: floor(max joint displacement / r) + 1."""
    import torch
    g = (edges[:, 1] - edges[:, 0]).abs().max().item() if edges.shape[0] else 0.0
    return int(np.floor(g / r)) + 1


def steer(robot: Robot, world: World, edges, n, stream=None):
    """cr_steer on edges (CUDA float32 [E, 2, dof]) with n + 1 samples each.
    Returns dict(last, v_new, dist, valid)."""
    import torch
    edges = edges.contiguous()
    E, D = edges.shape[0], edges.shape[2]
    dev = edges.device
    samples = torch.empty((E, n + 1, D), device=dev)
    valid = torch.empty((E, n + 1), device=dev, dtype=torch.uint8)
    cost = torch.empty((E, n + 1), device=dev)
    last = torch.empty(E, device=dev, dtype=torch.int32)
    v_new = torch.empty((E, D), device=dev)
    dist = torch.empty(E, device=dev)
    check(lib().cr_steer(robot.handle, world.handle, int(E), _dptr(edges), int(n), _dptr(samples),
                         _dptr(valid), _dptr(cost), _dptr(last), _dptr(v_new), _dptr(dist),
                         _stream(stream)), "cr_steer")
    return dict(last=last, v_new=v_new, dist=dist, valid=valid)


def retime(robot: Robot, problem: ProblemSpec, theta, stream=None):
    """dt that puts each trajectory of theta (CUDA float32 [B, H, dof]) at the
    robot's velocity, acceleration or jerk limit (cr_retime)."""
    import torch
    theta = theta.contiguous()
    dt = torch.empty(theta.shape[0], device=theta.device)
    pr = problem.struct()
    check(lib().cr_retime(robot.handle, C.byref(pr), int(theta.shape[0]), _dptr(theta), _dptr(dt),
                          _stream(stream)), "cr_retime")
    return dt


RANK_WEIGHTS = dict(w_pose=1.0, w_jerk=1e-3, w_time=1.0, w_dist=0.1)


def rank_seeds(robot: Robot, problem: ProblemSpec, theta, cfree, params=None, dt=None, stream=None,
               **weights):
    """Scores of the seeds theta (CUDA [B, H, dof]) and the index of the best
    collision-free one (App. "Solver details"; cr_rank_seeds).  IK mode in
    params: pose error + distance to q_start; else pose error, largest jerk at
    dt (CUDA [B], or params' dt) and motion time.  Weights default to
    RANK_WEIGHTS (the paper gives none).  Returns (score [B], best [1])."""
    import torch
    theta = theta.to(torch.float32).contiguous()
    if dt is not None:
        dt = dt.to(torch.float32).contiguous()
    B = theta.shape[0]
    w = dict(RANK_WEIGHTS)
    w.update(weights)
    P = params if isinstance(params, Params) else make_params(params)
    score = torch.empty(B, device=theta.device)
    best = torch.empty(1, device=theta.device, dtype=torch.int32)
    cf = cfree.contiguous().to(torch.uint8)
    pr = problem.struct()
    check(lib().cr_rank_seeds(robot.handle, C.byref(pr), C.byref(P), int(B), _dptr(theta), _dptr(cf),
                              _dptr(dt), float(w["w_pose"]),
                              float(w["w_jerk"]), float(w["w_time"]), float(w["w_dist"]), _dptr(score),
                              _dptr(best), _stream(stream)), "cr_rank_seeds")
    return score, best


class TimeoptOutput:
    """Device outputs of the stages of one problem's time-discretised solve."""

    def __init__(self, n_seeds, horizon, dof, device="cuda"):
        import torch
        self.first = torch.empty((horizon, dof), device=device)
        self.stage = torch.empty(8, device=device)
        self.dt = torch.empty(n_seeds, device=device)
        self.score = torch.empty(n_seeds, device=device)
        self.chosen = torch.empty(1, device=device, dtype=torch.int32)
        self._struct = TimeoptResult(_dptr(self.first), _dptr(self.stage), _dptr(self.dt), _dptr(self.score),
                                     _dptr(self.chosen))

    def struct(self) -> TimeoptResult:
        return self._struct


def time_discretized_solve(ctx, robot: Robot, problems, params=None, iters=(100, 100), dt_init=0.25,
                           dt_min=1e-3, w_pose=1.0, w_jerk=1e-3, w_time=1.0, graph=True, persistent=True,
                           stream=None):
    """Alg. "Time Discretization" through cr_solve_timeopt (every stage on the
    device, include/crgb.h).  problems: one ProblemSpec (host seeds) or a list.
    Returns, per problem, (SolveOutput of the second solve, TimeoptOutput)."""
    single = isinstance(problems, ProblemSpec)
    probs = [problems] if single else list(problems)
    n = len(probs)
    arr = (Problem * n)(*[p.struct() for p in probs])
    outs = [SolveOutput(p.struct().n_seeds, p.horizon, robot.dof) for p in probs]
    touts = [TimeoptOutput(p.struct().n_seeds, p.horizon, robot.dof) for p in probs]
    res = (Result * n)(*[o.struct() for o in outs])
    tres = (TimeoptResult * n)(*[o.struct() for o in touts])
    cfg = TimeoptConfig(float(dt_init), float(dt_min), int(iters[0]), int(iters[1]), float(w_pose),
                        float(w_jerk), float(w_time))
    P = params if isinstance(params, Params) else make_params(params)
    flags = (SOLVE_GRAPH if graph else 0) | (SOLVE_PERSISTENT if persistent else 0)
    check(lib().cr_solve_timeopt(ctx.handle, robot.handle, n, arr, C.byref(P), C.byref(cfg), flags, res, tres,
                                 _stream(stream)), "cr_solve_timeopt")
    pairs = list(zip(outs, touts))
    return pairs[0] if single else pairs


class OptBuffers:
    """Device-resident optimiser state of B seeds (cr_opt_state), as torch tensors."""

    def __init__(self, n_seeds, horizon, dof, history, n_alpha, device="cuda"):
        import torch
        B, n, m, na = n_seeds, horizon * dof, history, n_alpha
        z = lambda *s, dt=torch.float32: torch.zeros(s, device=device, dtype=dt)
        self.n_seeds, self.horizon, self.dof, self.m, self.na = B, horizon, dof, m, na
        self.x, self.g, self.c = z(B, n), z(B, n), z(B)
        self.x_prev, self.g_prev = z(B, n), z(B, n)
        self.s, self.y, self.rho = z(B, m, n), z(B, m, n), z(B, m)
        self.iter = z(B, dt=torch.int32)
        self.dir = z(B, n)
        self.cand, self.cand_cost = z(B, na, n), z(B, na)
        self.cand_grad = z(B, na, n)
        self.cand_cfree = z(B, na, dt=torch.uint8)
        self.best_x, self.best_c = z(B, n), z(B)
        self.best_cfree = z(B, dt=torch.uint8)
        self.ls_index = z(B, dt=torch.int32)

    def struct(self) -> OptState:
        f = [_dptr(getattr(self, k)) for k in
             ("x", "g", "c", "x_prev", "g_prev", "s", "y", "rho", "iter", "dir", "cand",
              "cand_cost", "cand_grad", "cand_cfree", "best_x", "best_c", "best_cfree",
              "ls_index")]
        return OptState(self.n_seeds, self.horizon, *f)


def opt_propose(robot: Robot, params, st: OptBuffers, stream=None):
    P = params if isinstance(params, Params) else make_params(params)
    s = st.struct()
    check(lib().cr_opt_propose(robot.handle, C.byref(P), C.byref(s), _stream(stream)),
          "cr_opt_propose")


def opt_select(robot: Robot, params, st: OptBuffers, stream=None):
    P = params if isinstance(params, Params) else make_params(params)
    s = st.struct()
    check(lib().cr_opt_select(robot.handle, C.byref(P), C.byref(s), _stream(stream)),
          "cr_opt_select")


# ---------------------------------------------------------------------------
# runtime
# ---------------------------------------------------------------------------

class Context:
    """Solver context on one device (workspace, captured graphs, autotune table)."""

    def __init__(self, device: int = 0, mem_budget: int = 0):
        h = _vp()
        check(lib().cr_context_create(int(device), int(mem_budget), C.byref(h)), "cr_context_create")
        self.handle = h
        self.device = device

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.cr_context_destroy(h)
            self.handle = None


class SolveOutput:
    """Device result buffers of one problem (torch tensors)."""

    def __init__(self, n_seeds, horizon, dof, device="cuda"):
        import torch
        self.traj = torch.empty((n_seeds, horizon, dof), device=device)
        self.cost = torch.empty(n_seeds, device=device)
        self.cfree = torch.empty(n_seeds, device=device, dtype=torch.uint8)
        self.best = torch.empty(1, device=device, dtype=torch.int32)
        self.status = torch.empty(1, device=device, dtype=torch.int32)
        self._struct = Result(_dptr(self.traj), _dptr(self.cost), _dptr(self.cfree), _dptr(self.best),
                              _dptr(self.status))

    def struct(self) -> Result:
        return self._struct


def solve(ctx: Context, robot: Robot, problems, params=None, iters=25, graph=True,
          persistent=True, outputs=None, stream=None, device_seeds=None, particles=None):
    """Optimise a batch of problems (ProblemSpec with host seeds) together.
    With device_seeds (one CUDA tensor [B, H, dof] per problem) the seeds are
    read from device memory instead.  particles: dict(iters, n_particles,
    beta, k_mu, k_sigma, sigma0, eps) runs particle-based optimisation of every
    seed first (cr_solve_particles; eps a CUDA tensor of iters x n_particles x
    V samples in that call's layout).  Returns one SolveOutput per problem
    (device tensors, valid once the stream has finished)."""
    probs = list(problems)
    n = len(probs)
    structs = [p.struct() for p in probs]
    if device_seeds is not None:
        structs = [Problem.from_buffer_copy(s) for s in structs]  # the cached views stay host-seeded
        for s, t in zip(structs, device_seeds):
            s.seeds = C.cast(C.c_void_p(t.data_ptr()), _fp)
            s.n_seeds = int(t.shape[0])
    arr = (Problem * n)(*structs)
    if outputs is None:
        outputs = [SolveOutput(s.n_seeds, p.horizon, robot.dof) for s, p in zip(structs, probs)]
    res = (Result * n)(*[o.struct() for o in outputs])
    P = params if isinstance(params, Params) else make_params(params)
    flags = (SOLVE_GRAPH if graph else 0) | (SOLVE_PERSISTENT if persistent else 0)
    if device_seeds is not None:
        flags |= SOLVE_DEVICE_SEEDS
    if particles is None:
        check(lib().cr_solve(ctx.handle, robot.handle, n, arr, C.byref(P), int(iters), flags, res,
                             _stream(stream)), "cr_solve")
        return outputs
    pc = ParticleConfig(int(particles["iters"]), int(particles["n_particles"]), float(particles["beta"]),
                        float(particles["k_mu"]), float(particles["k_sigma"]), float(particles["sigma0"]),
                        _dptr(particles["eps"].contiguous()))
    check(lib().cr_solve_particles(ctx.handle, robot.handle, n, arr, C.byref(P), int(iters), flags, C.byref(pc),
                                   res, _stream(stream)), "cr_solve_particles")
    return outputs


def evaluate_batch_noalloc(robot: Robot, problems, thetas, params=None, stream=None):
    """Evaluate several problems' trajectories in one launch through the entry
    point that allocates nothing on the device (the caller passes every input
    and output buffer).  thetas: one CUDA tensor [n_traj, H, dof] per problem.
    Returns per-problem dicts of cost / grad / cfree / terms (views into
    concatenated output tensors)."""
    import torch
    probs = list(problems)
    n = len(probs)
    arr = (Problem * n)(*[p.struct() for p in probs])
    counts = _i32([int(t.shape[0]) for t in thetas])
    theta = torch.cat([t.contiguous().view(-1) for t in thetas]).contiguous()
    T = int(counts.sum())
    dev = theta.device
    cost = torch.empty(T, device=dev)
    grad = torch.empty_like(theta)
    cfree = torch.empty(T, device=dev, dtype=torch.uint8)
    terms = torch.empty((T, N_TERMS), device=dev)
    P = params if isinstance(params, Params) else make_params(params)
    check(lib().cr_eval_batch_noalloc(robot.handle, n, arr, C.byref(P), _p(counts, _ip), _dptr(theta),
                                      _dptr(cost), _dptr(grad), _dptr(cfree), _dptr(terms),
                                      _stream(stream)), "cr_eval_batch_noalloc")
    out, t0, v0 = [], 0, 0
    for t in thetas:
        nt, nv = int(t.shape[0]), t.numel()
        out.append(dict(cost=cost[t0:t0 + nt], grad=grad[v0:v0 + nv].view(t.shape),
                        cfree=cfree[t0:t0 + nt], terms=terms[t0:t0 + nt]))
        t0 += nt
        v0 += nv
    return out


def autotune(ctx: Context, robot: Robot, problems, params=None, iters=2):
    """Measure the tile shapes on this batch and keep the fastest in ctx.
    Returns dict(block, short_tile, ms)."""
    probs = list(problems)
    arr = (Problem * len(probs))(*[p.struct() for p in probs])
    P = params if isinstance(params, Params) else make_params(params)
    bl, sh, nc, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_float()
    check(lib().cr_autotune(ctx.handle, robot.handle, len(probs), arr, C.byref(P), int(iters),
                            C.byref(bl), C.byref(sh), C.byref(nc), C.byref(ms)), "cr_autotune")
    return dict(block=bl.value, short_tile=sh.value, no_cache=nc.value, ms=ms.value)


def tune_set(ctx: Context, n_spheres, n_boxes, horizon, block, short_tile, no_cache=0):
    check(lib().cr_tune_set(ctx.handle, int(n_spheres), int(n_boxes), int(horizon), int(block),
                            int(short_tile), int(no_cache)), "cr_tune_set")


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------

class ServerConfig(C.Structure):
    _fields_ = [("kind_iters", C.c_int32 * 2), ("kind_params", Params * 2), ("chunk", C.c_int32),
                ("max_active", C.c_int32), ("reserve_bytes", C.c_size_t), ("max_queued", C.c_int32)]


MG, IK = 0, 1
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENAN = 0, 1, 2, 3, 4, 5, 6


class Server:
    """Continuous-batching server (cr_server_*): requests of two kinds and any
    shape, state resident on the device, admission by free device memory."""

    def __init__(self, ctx: Context, robot: Robot, mg_iters=100, ik_iters=50, mg_params=None, ik_params=None,
                 chunk=10, max_active=0, reserve_bytes=2 << 30, max_queued=0):
        cfg = ServerConfig()
        cfg.kind_iters[0], cfg.kind_iters[1] = mg_iters, ik_iters
        cfg.kind_params[0] = mg_params if isinstance(mg_params, Params) else make_params(mg_params)
        ikp = ik_params if ik_params is not None else dict(flags=IK_MODE | SELF | WOLFE)
        cfg.kind_params[1] = ikp if isinstance(ikp, Params) else make_params(ikp)
        cfg.chunk, cfg.max_active, cfg.reserve_bytes, cfg.max_queued = chunk, max_active, reserve_bytes, max_queued
        self.dof = robot.dof
        h = _vp()
        check(lib().cr_server_create(ctx.handle, robot.handle, C.byref(cfg), C.byref(h)),
              "cr_server_create")
        self.handle = h
        self._shape = {}

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.cr_server_destroy(h)
            self.handle = None

    def submit(self, kind, spec: ProblemSpec) -> int:
        pr = spec.struct()
        t = C.c_uint64()
        check(lib().cr_server_submit(self.handle, int(kind), C.byref(pr), C.byref(t)),
              "cr_server_submit")
        self._shape[t.value] = (int(pr.n_seeds), spec.horizon)
        return t.value

    def step(self, stream=None):
        check(lib().cr_server_step(self.handle, _stream(stream)), "cr_server_step")

    def poll(self, ticket):
        """None while pending, else dict(traj, cost, cfree, best, status) (host numpy)."""
        B, H = self._shape[ticket]
        done = C.c_int32()
        traj = np.empty((B, H, self.dof), dtype=np.float32)
        cost = np.empty(B, dtype=np.float32)
        cfree = np.empty(B, dtype=np.uint8)
        best, status = C.c_int32(), C.c_int32()
        check(lib().cr_server_poll(self.handle, int(ticket), C.byref(done), _p(traj), _p(cost),
                                   _p(cfree, _up), C.byref(best), C.byref(status)), "cr_server_poll")
        if not done.value:
            return None
        return dict(traj=traj, cost=cost, cfree=cfree.astype(bool), best=best.value, status=status.value)

    def wait(self, ticket, timeout_ms=-1):
        check(lib().cr_server_wait(self.handle, int(ticket), int(timeout_ms)), "cr_server_wait")
        return self.poll(ticket)

    def snapshot(self, ticket) -> bytes:
        n = C.c_size_t()
        check(lib().cr_server_snapshot(self.handle, int(ticket), None, C.byref(n)), "cr_server_snapshot")
        buf = C.create_string_buffer(n.value)
        check(lib().cr_server_snapshot(self.handle, int(ticket), buf, C.byref(n)), "cr_server_snapshot")
        return buf.raw[:n.value]

    def restore(self, blob: bytes, world: World) -> int:
        t = C.c_uint64()
        buf = C.create_string_buffer(blob, len(blob))
        check(lib().cr_server_restore(self.handle, buf, len(blob), world.handle, C.byref(t)), "cr_server_restore")
        hdr = np.frombuffer(blob[:48], dtype=np.int32)
        self._shape[t.value] = (int(hdr[3]), int(hdr[4]))   # B, H of the snapshot header
        return t.value

    def stats(self):
        a, q, b = C.c_int32(), C.c_int32(), C.c_size_t()
        check(lib().cr_server_stats(self.handle, C.byref(a), C.byref(q), C.byref(b)), "cr_server_stats")
        return dict(active=a.value, queued=q.value, pool_bytes=b.value)
