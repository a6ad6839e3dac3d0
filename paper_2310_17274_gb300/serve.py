"""Serving driver: a Poisson stream of motion-generation and IK requests
through the continuous-batching server (cr_server_*), and the same stream
through plain per-request solves, with p50 / p99 latency and throughput.

Requests are synthetic: motion generation = 32 seeds x 48 timesteps on a
world of 20-120 boxes, IK = 32 seeds on a 40-box world, goals from the
library's own forward kinematics of random configurations.
"""
from __future__ import annotations

import time

import numpy as np


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


def make_requests(crgb, synth, R, rb, n, seed=5, mg_shape=(32, 48), ik_seeds=32, n_worlds=16):
    """n requests, alternating kinds at random (1:1), with arrival order."""
    import torch
    rng = np.random.default_rng(seed)
    worlds = []
    for w in range(n_worlds):
        K = int(rng.integers(20, 121))
        worlds.append(crgb.World(synth.make_world(K, 1000 + w)))
    ik_world = crgb.World(synth.make_world(40, 999))
    qg = synth.uniform_config(rng, rb, n)
    _, ee, _ = crgb.fk(R, torch.tensor(qg, dtype=torch.float32, device="cuda"), spheres=False)
    ee = ee.cpu().numpy().astype(np.float64).reshape(-1, 3, 4)
    goals = [np.concatenate([e[:, 3], _rot_to_quat(e[:, :3])]) for e in ee]
    reqs = []
    B, H = mg_shape
    for i in range(n):
        if rng.random() < 0.5:
            qs = synth.uniform_config(rng, rb)
            seeds = synth.linear_seeds(rng, rb, qs, qg[i], B, H)
            spec = crgb.ProblemSpec(worlds[int(rng.integers(n_worlds))], qs, goals[i], H, seeds=seeds)
            reqs.append((crgb.MG, spec))
        else:
            seeds = synth.uniform_config(rng, rb, ik_seeds)[:, None, :]
            qs = synth.uniform_config(rng, rb)
            reqs.append((crgb.IK, crgb.ProblemSpec(ik_world, qs, goals[i], 1, seeds=seeds)))
    return reqs, worlds + [ik_world]


def poisson_arrivals(rate, n, seed=6):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def run_served(crgb, server, reqs, arrivals, horizon_s):
    """Feed requests at their arrival times; latency = completion - arrival."""
    t0 = time.perf_counter()
    pending = {}
    lat = np.full(len(reqs), np.nan)
    nxt = 0
    while True:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] <= now:
            pending[server.submit(*reqs[nxt])] = nxt
            nxt += 1
        if pending:
            server.step()
            done_t = time.perf_counter() - t0
            for t in list(pending):
                if server.poll(t) is not None:
                    i = pending.pop(t)
                    lat[i] = done_t - arrivals[i]
        elif nxt < len(reqs):
            time.sleep(max(0.0, min(arrivals[nxt] - now, 0.01)))
        if nxt >= len(reqs) and not pending:
            break
        if now > horizon_s:
            break
    wall = time.perf_counter() - t0
    while pending:   # finish what is left, untimed, so the server is empty again
        server.step()
        for t in list(pending):
            if server.poll(t) is not None:
                pending.pop(t)
    return lat, wall


def run_plain(crgb, ctx, R, reqs, arrivals, params, horizon_s):
    """Plain per-request path: one request at a time in arrival order, each a
    separate eager cr_solve (no batching, no graph)."""
    import torch
    t0 = time.perf_counter()
    lat = np.full(len(reqs), np.nan)
    for i, (kind, spec) in enumerate(reqs):
        now = time.perf_counter() - t0
        if now > horizon_s:
            break
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        p, iters = params[kind]
        out = crgb.solve(ctx, R, [spec], p, iters=iters, graph=False, persistent=False)[0]
        out.cost.cpu()
        torch.cuda.synchronize()
        lat[i] = time.perf_counter() - t0 - arrivals[i]
    return lat, time.perf_counter() - t0


def summarize(lat, arrivals, wall):
    """Percentiles over every offered request; one still unfinished when the
    run stopped counts with the time it had waited so far (a lower bound), so
    an overloaded path is not flattered."""
    done = np.isfinite(lat)
    filled = np.where(done, lat, wall - arrivals)
    if filled.size == 0:
        return {"offered": 0}
    return {"offered": int(filled.size), "completed": int(done.sum()),
            "p50_ms": float(np.percentile(filled, 50) * 1e3),
            "p99_ms": float(np.percentile(filled, 99) * 1e3),
            "throughput_req_s": float(done.sum() / wall), "wall_s": float(wall)}


def serving_benchmark(crgb, synth, ctx, R, rb, rates=(100.0, 250.0, 500.0), seconds=20.0, warm_s=2.0,
                      drain_s=5.0, chunk=10, mg_iters=100, ik_iters=50, max_active=64):
    """Continuous batching vs plain per-request solves on the same Poisson
    stream (MG:IK = 1:1) at each rate.  Both paths see the same arrivals
    over warm_s + seconds and may drain for drain_s more; requests arriving
    in the warm-up are not counted; one unfinished at the end counts with its
    wait so far (so an overloaded path reports a lower bound)."""
    mg_p = crgb.make_params(dict(alpha=list(synth.ALPHA_8)))
    ik_p = crgb.make_params(dict(flags=crgb.IK_MODE | crgb.SELF | crgb.WOLFE))
    params = {crgb.MG: (mg_p, mg_iters), crgb.IK: (ik_p, ik_iters)}
    # at most max_active requests per pool: beyond the device's capacity the
    # rest wait in the queue instead of slowing every round (and growing the
    # pools) for all
    server = crgb.Server(ctx, R, mg_iters=mg_iters, ik_iters=ik_iters, mg_params=mg_p, ik_params=ik_p,
                         chunk=chunk, max_active=max_active)
    out = {"seconds": seconds, "warmup_s": warm_s, "drain_s": drain_s, "chunk": chunk, "mix": "MG:IK = 1:1",
           "mg_iters": mg_iters, "ik_iters": ik_iters, "max_active_per_pool": max_active, "rates": []}
    warmed = False
    for k, rate in enumerate(rates):
        n = int(rate * (seconds + warm_s)) + 1
        reqs, keep = make_requests(crgb, synth, R, rb, n, seed=5 + k)
        arr = poisson_arrivals(rate, n, seed=6 + k)
        arr = arr[arr <= seconds + warm_s]
        reqs = reqs[:len(arr)]
        if not warmed:   # a few requests through both paths first
            w = min(8, len(reqs))
            run_served(crgb, server, reqs[:w], np.zeros(w), 60.0)
            run_plain(crgb, ctx, R, reqs[:w], np.zeros(w), params, 60.0)
            warmed = True
        horizon = seconds + warm_s + drain_s
        cnt = arr >= warm_s
        lat, wall = run_served(crgb, server, reqs, arr, horizon)
        served = summarize(lat[cnt], arr[cnt], wall)
        served["pool_bytes"] = server.stats()["pool_bytes"]
        lat_p, wall_p = run_plain(crgb, ctx, R, reqs, arr, params, horizon)
        plain = summarize(lat_p[cnt], arr[cnt], wall_p)
        out["rates"].append({"rate_req_s": rate, "served": served, "plain": plain})
        del keep
    return out
