#!/usr/bin/env python
"""Benchmark: seed x timestep cost+grad evaluations per second of the
trajectory-optimisation workload (7-DOF chain, 60 spheres, 32 boxes, 32 seeds
x 48 timesteps, 8 line-search step sizes, 100 L-BFGS iterations), one step =
one whole solve of that problem through the graph-captured batched path.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): independent replicas,
one problem per rank, max-over-ranks timing, value = total evaluations / time.
--impl reference times the FP64 CPU oracle (single-threaded) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "seed·timestep cost+grad evals/s"
UNIT = "evals/s"
WORKLOAD = ("trajopt: 7-DOF revolute chain, 60 spheres, 32 cuboids, 32 seeds x 48 timesteps, "
            "8 line-search step sizes, 100 L-BFGS iterations (history 6), FP32")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """Largest value over the ranks of the process group (itself alone when
    there is none): the whole job ends when its slowest replica does."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, steps: int, world_size: int, t_max: float) -> float:
    """Units of all replicas divided by the slowest replica's time."""
    return units_per_rank * steps * world_size / t_max


# ---------------------------------------------------------------------------
# workload (synthetic, seeded)
# ---------------------------------------------------------------------------

def start_config(synth, rb, seed_offset=0):
    """q_start of the trajectory workload, drawn from its own stream (the
    problem's stream, seed 2, draws q_goal)."""
    return synth.uniform_config(np.random.default_rng(1002 + seed_offset), rb)


def make_workload(crgb, synth, seed_offset=0):
    """Trajectory-optimisation problem; goal and box rejection through the
    library's own kinematics / evaluation (no oracle on this path)."""
    import torch
    cfg = synth.CONFIGS["trajopt"]
    rb = synth.make_robot(cfg.spheres_per_link, seed=0)
    R = crgb.Robot(rb)
    qs = start_config(synth, rb, seed_offset)

    def goal_fn(q):
        _, ee, _ = crgb.fk(R, torch.tensor(q, dtype=torch.float32, device="cuda")[None], spheres=False)
        E = ee[0].cpu().numpy().astype(np.float64).reshape(3, 4)
        return np.concatenate([E[:, 3], _rot_to_quat(E[:, :3])])

    ik_params = crgb.make_params(dict(flags=crgb.IK_MODE | crgb.SELF))

    def reject(pose, he):
        W1 = crgb.World(synth.World(pose=pose[None], half_ext=he[None]))
        spec = crgb.ProblemSpec(W1, qs, np.array([0, 0, 0, 1.0, 0, 0, 0]), 1)
        out = crgb.evaluate(R, spec, torch.tensor(qs, dtype=torch.float32, device="cuda").view(1, 1, -1),
                            ik_params, want_grad=False, want_terms=False)
        return not bool(out["cfree"][0])

    world = synth.make_world(cfg.n_boxes, cfg.world_seed + seed_offset, reject)
    pr = synth.make_problem(rb, world, 2 + seed_offset, cfg.n_seeds, cfg.horizon, goal_fn, q_start=qs)
    return cfg, rb, R, world, pr


def _rot_to_quat(R):
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
    q = np.asarray(q)
    return q / np.linalg.norm(q)


# DRAM bytes per launch of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, profiles/k_eval_trajopt_32x48x8.md),
# valid only for the kernel sources it was taken on: the key is the sha256 of
# those sources; any change to them reports traffic as null until recaptured.
EVAL_TRAFFIC = {"bytes": 652288, "states": 12288, "sources_sha256": "4620cd341a68e038",
                "profile": "profiles/k_eval_trajopt_32x48x8.md"}
EVAL_SOURCES = ("paper_2310_17274_gb300/csrc/k_eval.cu", "paper_2310_17274_gb300/csrc/crgb_internal.cuh",
                "paper_2310_17274_gb300/csrc/k_device.cuh", "paper_2310_17274_gb300/csrc/fastdiv.h")


def eval_traffic(states_per_launch):
    import hashlib
    h = hashlib.sha256()
    for f in EVAL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if not h.hexdigest().startswith(EVAL_TRAFFIC["sources_sha256"]):
        return None
    if states_per_launch != EVAL_TRAFFIC["states"]:
        return None
    return EVAL_TRAFFIC["bytes"]


def flop_per_state(dof, M, K, P):
    """Algorithmic FP32 work of one state's cost + gradient (FMA = 2 FLOP):
    kinematics 81/joint, sphere transform 18/sphere, box distance 35 per
    (sphere, box), pair distance 12 per pair, Jacobian-transpose 17 per
    (sphere, joint on its chain) with (dof+1)/2 joints on average, neighbour
    spheres for the sweep and the speed metric 50/sphere, stencils and bounds
    40/joint."""
    return 81 * dof + 18 * M + 35 * M * K + 12 * P + 17 * M * (dof + 1) / 2 + 50 * M + 40 * dof


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = f"/tmp/crgb_clocks_{os.getpid()}.csv"

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path) if l.strip()]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for k, n in enumerate(names):
                if r[5 + k].strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def _oracle_sample():
    """The trajectory workload as the oracle sees it, and its bounded sample:
    cost + gradient of 8 seeds' trajectories (8 x 48 states) of one
    line-search batch (32 seeds x 8 step sizes)."""
    import oracle
    from paper_2310_17274_gb300 import synth
    oracle.build()
    cfg = synth.CONFIGS["trajopt"]
    rb = synth.make_robot(cfg.spheres_per_link, seed=0)
    qs = start_config(synth, rb)
    world = synth.make_world(cfg.n_boxes, cfg.world_seed,
                             lambda p, h: oracle.start_collides_with_box(rb, qs, p, h))
    pr = synth.make_problem(rb, world, 2, cfg.n_seeds, cfg.horizon,
                            lambda q: oracle.goal_pose_from_fk(rb, q), q_start=qs)
    return rb, world, qs, pr.goal, pr.seeds[:8]


def _oracle_worker(job):
    """One host core: (warm-up evaluations, then `steps` evaluations or as
    many as fit in `seconds`).  Returns (evaluations, states each, elapsed)."""
    warmup, steps, seconds = job
    import oracle
    rb, world, qs, goal, sample = _oracle_sample()
    for _ in range(warmup):
        oracle.evaluate(rb, world, qs, goal, sample)
    n = 0
    t0 = time.perf_counter()
    while (steps and n < steps) or (not steps and time.perf_counter() - t0 < seconds):
        oracle.evaluate(rb, world, qs, goal, sample)
        n += 1
    return n, sample.shape[0] * sample.shape[1], time.perf_counter() - t0


def _oracle_all_cores(warmup, steps, seconds):
    """The oracle as it stands on every host core at once (independent
    processes, started with spawn: this process may already hold a CUDA
    context).  Returns (states/s, cores, evaluations, states per evaluation,
    slowest core's time)."""
    import multiprocessing as mp
    import oracle
    oracle.build()   # once, before the workers load it
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(warmup, steps, seconds)] * cores)
    n = sum(r[0] for r in res)
    per = res[0][1]
    t = max(r[2] for r in res)
    return n * per / t, cores, n, per, t


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    # each step: every host core evaluates the bounded sample once
    value, cores, n, per, t = _oracle_all_cores(args.warmup, args.steps, 0.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"per step, on each of {cores} cores: cost+grad of 8 seeds x "
                                       f"48 timesteps ({per} states)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(seconds=10.0):
    """The oracle as it stands on every host core, on a bounded sample."""
    value, cores, n, per, t = _oracle_all_cores(1, 0, seconds)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "per_core": value / cores,
            "sample": f"{n} x cost+grad of 8 seeds x 48 timesteps on {cores} processes "
                      f"({n * per} states, {t:.1f} s)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def profile_ik(crgb, synth, n):
    """N IK-mode evaluations of 128,000 uniformly drawn configurations of the
    60-sphere robot against a 40-box world, with gradients (the candidate
    batch of 1000 goals x 32 seeds x 4 step sizes), inside one NVTX range."""
    import torch
    cfg = synth.CONFIGS["ik"]
    rb = synth.make_robot(cfg.spheres_per_link, seed=0)
    R = crgb.Robot(rb)
    rng = np.random.default_rng(3)
    W = crgb.World(synth.make_world(cfg.n_boxes, cfg.world_seed))
    qs = synth.uniform_config(rng, rb)
    goal = np.array([0.3, 0.2, 0.5, 1.0, 0.0, 0.0, 0.0])
    q = torch.tensor(synth.uniform_config(rng, rb, 128000)[:, None, :], dtype=torch.float32, device="cuda")
    spec = crgb.ProblemSpec(W, qs, goal, 1)
    P = crgb.make_params(dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE))
    crgb.evaluate(R, spec, q, P, want_terms=False)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("crgb_eval_ik")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(n):
        crgb.evaluate(R, spec, q, P, want_terms=False)
    ev1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"profile_ik": n, "states_per_launch": 128000,
                      "us_per_launch": ev0.elapsed_time(ev1) / n * 1e3}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="crgb")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", default="ik,uneven,plain,serve,particle,linesearch,steer,timeopt")
    ap.add_argument("--serve-rates", default="100,250,500")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-warmup", type=float, default=2.0)
    ap.add_argument("--profile", type=int, default=0,
                    help="only run N fused evaluations of one line-search batch inside the NVTX "
                         "range crgb_eval (for ncu), then exit")
    ap.add_argument("--profile-ik", type=int, default=0,
                    help="only run N IK-mode evaluations of 128,000 states (40 boxes, self-collision, "
                         "gradients) inside the NVTX range crgb_eval_ik (for ncu), then exit")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    args.warmup = max(args.warmup, 3)

    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2310_17274_gb300 import build, crgb, synth
    if rank == 0 or not os.path.exists(crgb.LIB_PATH):
        build.build_library()
    if ws > 1:
        dist.barrier()

    if args.profile_ik:
        return profile_ik(crgb, synth, args.profile_ik)

    cfg, rb, R, world, pr = make_workload(crgb, synth, seed_offset=rank)
    W = crgb.World(world)
    B, H, D = pr.seeds.shape
    P = crgb.make_params(dict(alpha=list(cfg.alphas)))
    na = P.n_alpha
    iters = cfg.iters
    ctx = crgb.Context(local)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H, seeds=pr.seeds)
    seeds_dev = torch.tensor(pr.seeds, dtype=torch.float32, device="cuda")
    units = iters * B * na * H + B * H              # states evaluated per solve
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2

    if args.profile:
        cand = torch.tensor(np.repeat(pr.seeds, na, axis=0), dtype=torch.float32, device="cuda")
        espec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H)
        crgb.evaluate(R, espec, cand, P)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("crgb_eval")
        for _ in range(args.profile):
            crgb.evaluate(R, espec, cand, P, want_terms=False)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "states_per_launch": int(cand.shape[0] * H)}))
        return 0

    def solve_dev(outs=None):
        return crgb.solve(ctx, R, [spec], P, iters=iters, graph=True, persistent=True,
                          device_seeds=[seeds_dev], outputs=outs)

    outs = None
    for _ in range(args.warmup):
        outs = solve_dev(outs)
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM), L2 flushed between steps
    times = []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("crgb_step")
            ev0.record(stream)
            outs = solve_dev(outs)
            ev1.record(stream)
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
    clocks = clk.summary()
    t_total = max_over_ranks(float(np.sum(times)))
    value = whole_job_rate(units, args.steps, ws, t_total)
    launches_per_step = 2 + 2 * iters + 1

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    h_traj = torch.empty((B, H, D), dtype=torch.float32).pin_memory()
    h_cost = torch.empty(B, dtype=torch.float32).pin_memory()
    h_free = torch.empty(B, dtype=torch.uint8).pin_memory()
    h_best = torch.empty(1, dtype=torch.int32).pin_memory()
    e2e_times = []
    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = crgb.solve(ctx, R, [spec], P, iters=iters, graph=True, persistent=True, outputs=outs)[0]
        h_traj.copy_(o.traj, non_blocking=True)
        h_cost.copy_(o.cost, non_blocking=True)
        h_free.copy_(o.cfree, non_blocking=True)
        h_best.copy_(o.best, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    t_e2e = max_over_ranks(float(np.sum(e2e_times)))
    e2e_value = whole_job_rate(units, args.steps, ws, t_e2e)
    h2d = pr.seeds.size * 4
    d2h = h_traj.numel() * 4 + h_cost.numel() * 4 + h_free.numel() + h_best.numel() * 4

    # ---- dominant kernel: the fused evaluation of one line-search batch,
    # timed alone with CUDA events on its stream
    cand = torch.tensor(np.repeat(pr.seeds, na, axis=0), dtype=torch.float32, device="cuda")
    espec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H)
    for _ in range(5):
        crgb.evaluate(R, espec, cand, P)
    n_ev = 50
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(n_ev):
        crgb.evaluate(R, espec, cand, P, want_terms=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_eval = ev0.elapsed_time(ev1) / 1e3 / n_ev
    fps = flop_per_state(D, rb.n_spheres, world.n, rb.n_pairs)
    states_per_launch = B * na * H
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    derived = n_sm * 128 * 2 * sm_max * 1e6 / 1e12   # FP32 FMA lanes x 2 FLOP x clock
    # the measured FP32 FMA peak (the library's own microbenchmark, ~0.5 s)
    # with the SM clock sampled while it runs
    with Clocks(local) as pclk:
        peak_tflops, peak_ms = crgb.measure_ffma(iters=400000)
    pclocks = pclk.summary()
    achieved = fps * states_per_launch / t_eval / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": eval_traffic(states_per_launch),
                "traffic_source": EVAL_TRAFFIC["profile"], "kernel": "k_eval",
                "launch_us": t_eval * 1e6, "states_per_launch": states_per_launch,
                "flop_per_state": fps,
                "peak_note": f"measured FP32 FMA peak (cr_measure_ffma, {peak_ms:.0f} ms, median SM clock "
                             f"{pclocks.get('sm_mhz')} MHz); derived {n_sm} SMs x 128 lanes x 2 FLOP x "
                             f"{sm_max:.0f} MHz = {derived:.1f} TFLOP/s",
                "peak_derived": derived, "frac_of_derived": achieved / derived}

    extras = {}
    want = set(args.extras.split(",")) if args.extras else set()
    if rank == 0 and "plain" in want:
        # plain per-problem GPU path: eager launches, no graph, grid-strided tiles
        for _ in range(2):
            crgb.solve(ctx, R, [spec], P, iters=iters, graph=False, persistent=False,
                       device_seeds=[seeds_dev], outputs=outs)
        torch.cuda.synchronize()
        tp = []
        for _ in range(5):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            crgb.solve(ctx, R, [spec], P, iters=iters, graph=False, persistent=False,
                       device_seeds=[seeds_dev], outputs=outs)
            e1.record(stream)
            torch.cuda.synchronize()
            tp.append(e0.elapsed_time(e1) / 1e3)
        extras["plain_gpu_path"] = {"value": units / float(np.mean(tp)), "unit": UNIT,
                                    "ms_per_solve": float(np.mean(tp)) * 1e3,
                                    "what": "same solve, eager launches, no CUDA graph"}
    if rank == 0 and "ik" in want:
        extras["ik"] = bench_ik(crgb, synth, ctx, R, rb)
        extras["ik_particles"] = bench_ik(crgb, synth, ctx, R, rb, particle_iters=2)
        extras["ik_no_collision"] = bench_ik(crgb, synth, ctx, R, rb, collision=False)
    if rank == 0 and "particle" in want:
        extras["particle"] = bench_particle(crgb, synth, ctx, R, rb, world, pr, P, iters)
    if rank == 0 and "linesearch" in want:
        extras["line_search"] = bench_line_search(crgb, synth, ctx, R, world, pr, iters)
    if rank == 0 and "steer" in want:
        extras["steer"] = bench_steer(crgb, synth, R, rb, world)
    if rank == 0 and "timeopt" in want:
        extras["timeopt"] = bench_timeopt(crgb, synth, ctx, R, world, pr, dict(alpha=list(cfg.alphas)))
    if rank == 0 and "uneven" in want:
        extras["uneven"] = bench_uneven(crgb, synth, ctx, R, rb)
    if rank == 0 and "serve" in want:
        from paper_2310_17274_gb300 import serve
        rates = tuple(float(r) for r in args.serve_rates.split(","))
        extras["serve"] = serve.serving_benchmark(crgb, synth, ctx, R, rb, rates=rates,
                                                  seconds=args.serve_seconds, warm_s=args.serve_warmup)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "solve": "graph-captured, persistent evaluation",
                           "units_per_step": units, "parallelism": f"replicas x{ws}",
                           "l2": "flushed between steps (256 MB write)"},
                "clocks": clocks,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h),
                        "what": "cr_solve with host seeds, results read back to pinned host memory"},
                "gpu_launches": launches_per_step * args.steps,
                "roofline": roofline,
                "cpu_baseline": cpu,
                "extras": extras}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def bench_ik(crgb, synth, ctx, R, rb, n_goals=1000, n_seeds=32, iters=50, collision=True, particle_iters=0,
             n_particles=16, sigma0=0.01):
    """Batched IK: 1000 goals x 32 seeds (H = 1) in one solve.  With
    collision: 40 cuboids, self-collision on, goals from FK of collision-free
    configurations; without: no cuboids, no self term and no self check in
    the collision-free flag (the paper's IK without collision checking).
    Solved (Sec. 6's 5 mm / 5 % test): the best seed is collision-free, within
    5 mm, and its orientation distance d_q = (3 - tr(R_g^T R)) / 4 of Eq. 14 is
    at most 1e-3 (about 3.6 degrees); the looser reading d_q <= 0.05 (5 % of
    the [0, 1] range of d_q) is reported beside it."""
    import torch
    cfg = synth.CONFIGS["ik"]
    rng = np.random.default_rng(3)
    qs = synth.uniform_config(rng, rb)
    flags = crgb.IK_MODE | crgb.WOLFE | (crgb.SELF if collision else 0)
    # goals and box rejection use the full validity check (self-collision
    # included); the plain solve checks no collision at all (Sec. 6)
    checkp = crgb.make_params(dict(flags=flags, alpha=list(cfg.alphas)))
    ikp = crgb.make_params(dict(flags=flags | (0 if collision else crgb.NO_SELF_CHECK), alpha=list(cfg.alphas)))

    def reject(pose, he):
        W1 = crgb.World(synth.World(pose=pose[None], half_ext=he[None]))
        spec = crgb.ProblemSpec(W1, qs, np.array([0, 0, 0, 1.0, 0, 0, 0]), 1)
        out = crgb.evaluate(R, spec, torch.tensor(qs, dtype=torch.float32, device="cuda").view(1, 1, -1),
                            checkp, want_grad=False, want_terms=False)
        return not bool(out["cfree"][0])

    world = synth.make_world(cfg.n_boxes if collision else 0, cfg.world_seed, reject)
    W = crgb.World(world)
    # reachable goals: FK of configurations sampled within the limits, kept
    # (with collision) when the library's own check finds them free
    probe = crgb.ProblemSpec(W, qs, np.array([0, 0, 0, 1.0, 0, 0, 0]), 1)
    qg = np.zeros((0, rb.dof))
    while len(qg) < n_goals:
        cand = synth.uniform_config(rng, rb, 4096)
        ev = crgb.evaluate(R, probe, torch.tensor(cand[:, None, :], dtype=torch.float32, device="cuda"),
                           checkp, want_grad=False, want_terms=False)
        qg = np.concatenate([qg, cand[ev["cfree"].cpu().numpy().astype(bool)]])
    qg = qg[:n_goals]
    _, ee, _ = crgb.fk(R, torch.tensor(qg, dtype=torch.float32, device="cuda"), spheres=False)
    ee = ee.cpu().numpy().astype(np.float64).reshape(-1, 3, 4)
    goals = np.stack([np.concatenate([e[:, 3], _rot_to_quat(e[:, :3])]) for e in ee])
    seeds = synth.uniform_config(rng, rb, n_goals * n_seeds).reshape(n_goals, n_seeds, 1, rb.dof)
    specs = [crgb.ProblemSpec(W, qs, goals[g], 1, seeds=seeds[g]) for g in range(n_goals)]
    choice = crgb.autotune(ctx, R, specs, ikp, iters=5)
    # particle iterations before L-BFGS (App. B.3), from unit Gaussian samples
    # drawn on the device with a fixed generator seed
    pcfg = None
    if particle_iters > 0:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(321)
        eps = torch.randn(particle_iters * n_particles * n_goals * n_seeds * rb.dof, device="cuda", generator=gen)
        pcfg = dict(iters=particle_iters, n_particles=n_particles, beta=1000.0, k_mu=0.9, k_sigma=0.9,
                    sigma0=sigma0, eps=eps)
    outs = None
    for _ in range(3):
        outs = crgb.solve(ctx, R, specs, ikp, iters=iters, graph=True, persistent=True, outputs=outs,
                          particles=pcfg)
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        outs = crgb.solve(ctx, R, specs, ikp, iters=iters, graph=True, persistent=True, outputs=outs,
                          particles=pcfg)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    t = float(np.median(ts))
    Rg = np.stack([_quat_rot(g[3:]) for g in goals])

    def judge(pick):
        """Success of the seed `pick` of every goal, with the library's own kinematics."""
        best = torch.stack([o.traj[int(k), 0] for o, k in zip(outs, pick)])
        free = np.array([bool(o.cfree[int(k)]) for o, k in zip(outs, pick)])
        _, eb, _ = crgb.fk(R, best.contiguous(), spheres=False)
        eb = eb.cpu().numpy().astype(np.float64).reshape(-1, 3, 4)
        pos_err = np.linalg.norm(eb[:, :, 3] - goals[:, :3], axis=1)
        dq = (3 - np.einsum("nij,nij->n", Rg, eb[:, :, :3])) / 4
        ok = free if collision else np.ones_like(free)   # plain IK: pose only
        return free, pos_err, dq, ok & (pos_err <= 5e-3) & (dq <= 1e-3), ok & (pos_err <= 5e-3) & (dq <= 0.05)

    # the solve's best seed (lowest cost, collision-free first) ...
    free, pos_err, dq, solved, loose = judge([int(o.best) for o in outs])
    # ... and the seed App. "Solver details" returns for IK: the lowest pose
    # error + 0.1 x distance from the start among the collision-free seeds
    # (cr_rank_seeds on the device; the solve's best when none is free)
    t0 = time.perf_counter()
    picks = []
    for o, sp in zip(outs, specs):
        _, b = crgb.rank_seeds(R, sp, o.traj, o.cfree, ikp)
        picks.append(b)
    picks = [int(b) if int(b) >= 0 else int(o.best) for b, o in zip(picks, outs)]
    t_rank = time.perf_counter() - t0
    _, _, dq_r, solved_r, loose_r = judge(picks)
    return {"ik_solves_per_s": float(solved.sum()) / t, "ik_goals_per_s": n_goals / t,
            "success_rate": float(solved.mean()),
            "success": ("collision-free, " if collision else "") + "position within 5 mm, d_q <= 1e-3 "
                       "(the solve's best seed: lowest cost among the collision-free seeds)",
            "goals": n_goals, "seeds": n_seeds, "iters": iters, "boxes": int(world.n),
            "self_collision": bool(collision), "ms_per_batch": t * 1e3,
            "ik_solves_per_s_dq_0.05": float(loose.sum()) / t,
            "success_rate_dq_0.05": float(loose.mean()),
            "solver_details_choice": {
                "what": "the seed App. 'Solver details' returns for IK (cr_rank_seeds: lowest pose error + "
                        "0.1 x joint distance from the start among the collision-free seeds)",
                "success_rate": float(solved_r.mean()), "ik_solves_per_s": float(solved_r.sum()) / t,
                "success_rate_dq_0.05": float(loose_r.mean()), "median_dq": float(np.median(dq_r)),
                "choice_ms_host": t_rank * 1e3},
            "best_seed_collision_free": float(free.mean()),
            "within_5mm": float((pos_err <= 5e-3).mean()),
            "median_pos_err_m": float(np.median(pos_err)), "median_dq": float(np.median(dq)),
            "evals_per_s": n_goals * n_seeds * (iters * ikp.n_alpha + 1) / t,
            "goals_from": "FK of configurations sampled within the limits"
                          + (" (collision-free)" if collision else ""),
            "particle_iters": particle_iters,
            "particles": (f"{n_particles} per seed, sigma0 {sigma0}, beta 1000, k_mu = k_sigma = 0.9, "
                          "unit Gaussian samples") if particle_iters else None,
            "autotune": choice}


def _quat_rot(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def bench_particle(crgb, synth, ctx, R, rb, world, pr, P, iters, n_particles=16, n_iters=2,
                   beta=1000.0, k_mu=0.9, k_sigma=0.9, sigma0=0.01):
    """Sec. 4.2: n_iters particle iterations (n_particles per seed) before the
    L-BFGS solve of the trajectory workload, against the same solve from the
    raw seeds: time and final best costs.  The samples are drawn on the device
    from a fixed generator seed as smooth perturbations: a unit Gaussian
    offset per joint ramped linearly from 0 at the start to 1 at the last
    timestep (independent noise per timestep would make every particle
    jerky; the paper does not say how it samples)."""
    import torch
    B, H, D = pr.seeds.shape
    W = crgb.World(world)
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(123)
    ramp = torch.arange(1, H + 1, device="cuda", dtype=torch.float32).view(1, 1, 1, H, 1) / H
    eps = (torch.randn((n_iters, B, n_particles, 1, D), device="cuda", generator=gen) * ramp).contiguous()
    eps = eps.expand(n_iters, B, n_particles, H, D).contiguous()
    sspec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H, seeds=pr.seeds)
    cfg = dict(iters=n_iters, n_particles=n_particles, beta=beta, k_mu=k_mu, k_sigma=k_sigma, sigma0=sigma0,
               eps=eps)

    def run(particles):
        # one graph-captured cr_solve_particles call: particle iterations, then L-BFGS
        return crgb.solve(ctx, R, [sspec], P, iters=iters, graph=True, persistent=True,
                          particles=cfg if particles else None)[0]

    out = {}
    for particles in (False, True):
        for _ in range(2):
            run(particles)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        o = run(particles)
        e1.record()
        torch.cuda.synchronize()
        c = o.cost.cpu().numpy()
        f = o.cfree.cpu().numpy().astype(bool)
        out["particle+lbfgs" if particles else "lbfgs"] = {
            "ms": e0.elapsed_time(e1), "best_cost": float(c[int(o.best)]),
            "median_seed_cost": float(np.median(c)), "collision_free_seeds": int(f.sum())}
    out.update({"particles_per_seed": n_particles, "particle_iters": n_iters, "beta": beta,
                "k_mu": k_mu, "k_sigma": k_sigma, "sigma0": sigma0,
                "samples": "unit Gaussian end offset per joint, ramped linearly over the horizon"})
    return out


def bench_line_search(crgb, synth, ctx, R, world, pr, iters):
    """Line-search variants of Sec. 7.3 on the trajectory workload (same seeds,
    same iterations): noisy-ls (the default), noisy-ls-1, Wolfe and strong
    Wolfe over 12 step sizes with a 0.0 fallback, and no line search."""
    import torch
    W = crgb.World(world)
    B, H, D = pr.seeds.shape
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H, seeds=pr.seeds)
    wolfe12 = [0.0, 1e-4, 1e-3, 0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9, 1.0]
    base = crgb.params_default()["flags"] & ~(crgb.WOLFE | crgb.STRONG_WOLFE)
    variants = {
        "noisy-ls": dict(alpha=[0.01, 0.3, 0.7, 1.0], flags=base | crgb.WOLFE),
        "noisy-ls-1": dict(alpha=[0.01, 1.0], flags=base | crgb.WOLFE),
        "wolfe": dict(alpha=wolfe12, flags=base | crgb.WOLFE),
        "st-wolfe": dict(alpha=wolfe12, flags=base | crgb.WOLFE | crgb.STRONG_WOLFE),
        "no-ls": dict(alpha=[1.0], flags=base),
    }
    out = {}
    for name, p in variants.items():
        P = crgb.make_params(p)
        o = None
        for _ in range(2):
            o = crgb.solve(ctx, R, [spec], P, iters=iters, graph=True, persistent=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        o = crgb.solve(ctx, R, [spec], P, iters=iters, graph=True, persistent=True)[0]
        e1.record()
        torch.cuda.synchronize()
        c = o.cost.cpu().numpy()
        f = o.cfree.cpu().numpy().astype(bool)
        out[name] = {"step_sizes": len(p["alpha"]), "ms": e0.elapsed_time(e1),
                     "best_cost": float(c[int(o.best)]), "median_seed_cost": float(np.median(c)),
                     "collision_free_seeds": int(f.sum())}
    return out


def bench_steer(crgb, synth, R, rb, world, n_edges=4096, r=0.05):
    """Sec. 5 parallel steering: n_edges random edges (ends within the limits,
    joint steps N(0, 0.6^2)) in the trajectory workload's world, n + 1
    samples each at resolution r: edges and samples checked per second."""
    import torch
    rng = np.random.default_rng(12)
    a = synth.uniform_config(rng, rb, n_edges)
    b = np.clip(a + rng.normal(0, 0.6, size=a.shape), rb.q_lo, rb.q_hi)
    ed = torch.tensor(np.stack([a, b], axis=1), dtype=torch.float32, device="cuda")
    n = crgb.steer_steps(ed, r)
    W = crgb.World(world)
    for _ in range(3):
        out = crgb.steer(R, W, ed, n)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        out = crgb.steer(R, W, ed, n)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / 10
    last = out["last"].cpu().numpy()
    return {"edges": n_edges, "samples_per_edge": n + 1, "ms": t * 1e3, "edges_per_s": n_edges / t,
            "samples_per_s": n_edges * (n + 1) / t, "fully_valid_edges": int((last == n).sum()),
            "start_invalid_edges": int((last < 0).sum())}


def bench_timeopt(crgb, synth, ctx, R, world, pr, P_over):
    """Alg. "Time Discretization" on the trajectory workload through
    cr_solve_timeopt: solve at dt 0.25 without jerk, retime the best seed,
    scale the weights, solve again with jerk, retime and score every seed,
    all stages on the device in one CUDA graph."""
    import torch
    W = crgb.World(world)
    B, H, D = pr.seeds.shape
    spec = crgb.ProblemSpec(W, pr.q_start, pr.goal, H, seeds=pr.seeds)
    for _ in range(2):
        crgb.time_discretized_solve(ctx, R, spec, P_over, iters=(100, 100))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out, to = crgb.time_discretized_solve(ctx, R, spec, P_over, iters=(100, 100))
    e1.record()
    torch.cuda.synchronize()
    c = out.cost.cpu().numpy()
    st = to.stage.cpu().numpy()
    chosen = int(to.chosen)
    dt_f = float(to.dt[chosen])
    return {"ms": e0.elapsed_time(e1), "dt_opt": float(st[4]), "dt_final": dt_f, "motion_time_s": H * dt_f,
            "chosen_seed": chosen, "chosen_cost": float(c[chosen]), "best_cost": float(c[int(out.best)]),
            "collision_free_seeds": int(out.cfree.cpu().numpy().astype(bool).sum()),
            "what": "two 100-iteration solves (dt 0.25 without jerk, then dt_opt), every seed retimed, "
                    "the seed chosen by the blend of pose error, largest jerk and motion time; one "
                    "cr_solve_timeopt call, no host round trip between the stages (CUDA events)"}


def bench_uneven(crgb, synth, ctx, R, rb, iters=100):
    """64 problems with uneven box counts, seeds and horizons in one
    persistent graph-captured solve, against 64 separate plain solves."""
    import torch
    shapes = synth.uneven_shapes(4, 64)
    rng = np.random.default_rng(4)
    specs, worlds, units = [], [], 0
    for k, (K, B, H) in enumerate(shapes):
        world = synth.make_world(K, 400 + k)
        W = crgb.World(world)
        worlds.append(W)
        qs = synth.uniform_config(rng, rb)
        qg = synth.uniform_config(rng, rb)
        seeds = synth.linear_seeds(rng, rb, qs, qg, B, H)
        goal = np.array([0.3, 0.2, 0.5, 1, 0, 0, 0.0])
        specs.append(crgb.ProblemSpec(W, qs, goal, H, seeds=seeds))
        units += iters * B * 4 * H + B * H
    P = crgb.make_params(None)
    # tile shapes for these problem shapes from the autotuner (untimed)
    choice = crgb.autotune(ctx, R, specs, P, iters=10)
    outs = None
    for _ in range(2):
        outs = crgb.solve(ctx, R, specs, P, iters=iters, graph=True, persistent=True, outputs=outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        outs = crgb.solve(ctx, R, specs, P, iters=iters, graph=True, persistent=True, outputs=outs)
    e1.record()
    torch.cuda.synchronize()
    t_batched = e0.elapsed_time(e1) / 1e3 / 3
    # plain: 64 separate eager solves
    single = [None] * len(specs)
    for k, s in enumerate(specs):
        single[k] = crgb.solve(ctx, R, [s], P, iters=iters, graph=False, persistent=False)
    torch.cuda.synchronize()
    e0.record()
    for k, s in enumerate(specs):
        crgb.solve(ctx, R, [s], P, iters=iters, graph=False, persistent=False, outputs=single[k])
    e1.record()
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1e3
    same = all(torch.equal(a.cost, b[0].cost) for a, b in zip(outs, single))
    return {"problems": len(specs), "iters": iters, "evals_per_step": units,
            "batched_ms": t_batched * 1e3, "batched_evals_per_s": units / t_batched,
            "plain_ms": t_plain * 1e3, "plain_evals_per_s": units / t_plain,
            "speedup": t_plain / t_batched, "results_identical": bool(same),
            "autotune": choice}


if __name__ == "__main__":
    sys.exit(main())
