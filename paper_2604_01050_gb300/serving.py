"""Request loop over the batching engine: Poisson arrivals, p50/p99 latency.

A request is one Ising instance to solve (an SK +-1 instance or a 3D cubic
lattice spin glass, N between 64 and 8192, P in {8, 16, 32} replicas, R = 16
auto-tuned runs, a fixed step budget).  Requests arrive as a Poisson stream;
the loop submits every request whose arrival time has passed, advances the
engine by one chunk of steps (continuous batching: requests join and leave at
chunk boundaries while others keep running) and records, per request, the
time from arrival to the moment its result is on the host.

Instances come from a small pool generated up front (their couplings are
uploaded once, as a server caching its problem library would); requests
sample an instance, a replica count and a seed.
"""
from __future__ import annotations

import time

import numpy as np

from . import _binding as sb


def make_pool(n_instances=12, seed=0, n_min=64, n_max=8192, R=16):
    """Problem handles of mixed kind and size, each with its schedule set."""
    import workloads
    rng = np.random.default_rng(seed)
    pool = []
    for k in range(n_instances):
        n = int(rng.integers(n_min, n_max + 1))  # N uniform in [n_min, n_max]
        beta, alpha = workloads.autotune_params(R, seed + k)
        if k % 2 == 0:
            J, _ = workloads.sk_pm1(n, seed + k)
            pb = sb.create_problem_dense(J)
            kind = "sk"
        else:
            L = max(3, int(round(n ** (1.0 / 3.0))))
            nn, rp, col, val, h = workloads.cubic_lattice(L, seed + k)
            pb = sb.create_problem_csr(nn, rp, col, val, h)
            n, kind = nn, "lattice"
        sb.set_schedule(pb, beta, alpha)
        pool.append({"problem": pb, "n": n, "kind": kind})
    return pool


def make_requests(pool, n_requests, steps=2000, R=16, seed=1):
    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n_requests):
        inst = pool[int(rng.integers(len(pool)))]
        P = int(rng.choice([8, 16, 32]))
        reqs.append({"inst": inst, "P": P, "R": R, "steps": steps, "seed": int(rng.integers(1 << 62))})
    return reqs


def run_stream(reqs, rate, arena_bytes=40 << 30, slots=64, chunk=100, seed=2, stream=None, dense_batching=True):
    """Open loop at `rate` requests/s (closed loop, all at t = 0, if rate is
    None).  Returns per-request latencies (s), the makespan and the
    replica-spin updates done.  dense_batching: small dense requests share
    cooperative launches (sbqa_engine_set_dense_batching)."""
    rng = np.random.default_rng(seed)
    if rate is None:
        arrivals = np.zeros(len(reqs))
    else:
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    eng = sb.engine_create(arena_bytes, slots, chunk)
    sb.engine_set_dense_batching(eng, dense_batching)
    id_of = {}
    done_at = {}
    t0 = time.perf_counter()
    nxt = 0
    while len(done_at) < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] <= now:
            r = reqs[nxt]
            rid = sb.engine_submit(eng, r["inst"]["problem"], r["steps"], r["P"], r["R"], r["seed"])
            id_of[rid] = nxt
            nxt += 1
        st = sb.engine_stats(eng)
        if st["active"] == 0 and st["queued"] == 0:
            if nxt < len(reqs):
                time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
            continue
        for rid in sb.engine_step(eng, stream):
            done_at[id_of[rid]] = time.perf_counter() - t0
    makespan = time.perf_counter() - t0
    lat = np.array([done_at[q] - arrivals[q] for q in range(len(reqs))])
    updates = sum(r["inst"]["n"] * r["P"] * r["R"] * r["steps"] for r in reqs)
    results = {rid: sb.engine_result(eng, rid) for rid in id_of}
    stats = sb.engine_stats(eng)
    eng.destroy()
    return {"latency_s": lat, "makespan_s": makespan, "updates": updates, "results": results,
            "arrivals": arrivals, "kernels_launched": stats["kernels_launched"],
            "batched_updates": stats["batched_updates"], "batched_ms": stats["batched_ms"],
            "dense_batched_launches": stats["dense_batched_launches"],
            "dense_batched_chunks": stats["dense_batched_chunks"]}


def summary(out):
    lat = out["latency_s"]
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max()),
            "updates_per_s": out["updates"] / out["makespan_s"], "makespan_s": out["makespan_s"],
            "requests": int(lat.size), "kernels_launched": int(out["kernels_launched"]),
            "dense_batched_launches": int(out.get("dense_batched_launches", 0)),
            "dense_batched_chunks": int(out.get("dense_batched_chunks", 0))}
