#!/usr/bin/env python
"""Benchmark of the SBQA hot path (replica-spin updates/s) on GB300.

One benchmark step = one whole solve of the headline workload: initial
state, 5000 steps of the SBQA equations of motion on a random 6-regular graph
(N=10^5, J ~ N(0,1), h ~ N(0, 0.1^2), CSR, BF16 couplings) with P=16 Trotter
replicas and R=8 auto-tuned runs, then the readout (sign, energies of all 128
replicas, best per run).  Its state (128 MB) exceeds the L2 cache, so every
step streams it through HBM.  The same line carries ``per_config`` records,
measured the same way, of the 3D cubic lattice L=16 (N=4096, P=32, R=64,
10^4 steps), the dense SK N=2000 instance on the tensor cores (P=32, R=32,
1000 steps), the same shape with real Gaussian couplings on the BF16 tensor
cores, and the Poisson serving stream (p50/p99 latency).

  value   updates/s = N * P * R * steps / solve time, with J resident on the
          device (CUDA events on the library's stream; L2 flushed before every
          timed solve)
  e2e     the same metric through the C ABI from host buffers: create the
          problem from pinned host arrays, set the schedule, run, read the best
          result back, destroy -- all inside the timed region
  roofline  the step kernel against the measured HBM copy bandwidth, with the
          algorithmic 16 bytes per replica-spin update (x, y read + write),
          or, for the dense tensor-core kernels, 2 N^2 R P flops per step
          against the measured dense GEMM peak of their operand type

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload instead (rank 0 only).  Under torchrun every rank solves its own
copy of the workload (independent runs, no collective on the data path) and
``value`` is the total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

CONFIGS = {
    "lattice16": dict(kind="lattice", L=16, P=32, R=64, S=10000, prec="auto",
                      workload="3D cubic lattice spin glass L=16 (N=4096), periodic, J=+-1, CSR; "
                               "P=32 replicas, R=64 runs, 10^4 steps; FP32 state, exact int8 product"),
    "sk64": dict(kind="sk", n=64, P=8, R=16, S=1000, prec="auto",
                 workload="dense SK N=64, J=+-1, h=0; P=8, R=16, 1000 steps, linear schedule"),
    "sk2000": dict(kind="sk", n=2000, P=32, R=32, S=1000, prec="exact",
                   workload="dense SK N=2000, J=+-1; P=32, R=32 (J.X = 2000x2000 @ 2000x1024), 1000 steps"),
    # real-valued dense couplings (Gaussian SK): the BF16 tensor-core product
    "skreal2000": dict(kind="skreal", n=2000, P=32, R=32, S=1000, prec="bf16",
                       workload="dense SK N=2000, J~N(0,1), h~N(0,0.1^2), BF16 J on the tensor cores; P=32, R=32 "
                                "(J.X = 2000x2000 @ 2000x1024), 1000 steps"),
    "regular1e5": dict(kind="regular", n=100000, d=6, P=16, R=8, S=5000, prec="bf16",
                       workload="random 6-regular N=1e5, J~N(0,1), h~N(0,0.1^2), CSR, BF16 J, P=16, R=8, 5000 steps"),
    # large-N sparse family: the lattice16 shape (P=32, R=64) as the state outgrows L2
    "regular7e5": dict(kind="regular", n=700000, d=6, P=16, R=8, S=1000, prec="bf16",
                       workload="random 6-regular N=7e5, J~N(0,1), h~N(0,0.1^2), CSR, BF16 J, P=16, R=8, 1000 steps"),
}
for _L, _S in ((24, 3000), (32, 1500), (48, 400), (64, 200), (88, 100)):
    CONFIGS["lattice%d" % _L] = dict(
        kind="lattice", L=_L, P=32, R=64, S=_S, prec="auto",
        workload="3D cubic lattice spin glass L=%d (N=%d), periodic, J=+-1, CSR; P=32 replicas, R=64 runs, "
                 "%d steps; FP32 state, exact int8 product" % (_L, _L ** 3, _S))
for _n, _S in ((4096, 500), (8192, 200)):
    CONFIGS["sk%d" % _n] = dict(
        kind="sk", n=_n, P=32, R=32, S=_S, prec="exact",
        workload="dense SK N=%d, J=+-1; P=32, R=32 (J.X = %dx%d @ %dx1024), %d steps" % (_n, _n, _n, _n, _S))
# a tall dense instance (many spins, few replica columns): the persistent solver splits its K loop
CONFIGS["sk8192t"] = dict(kind="sk", n=8192, P=8, R=32, S=200, prec="exact",
                          workload="dense SK N=8192, J=+-1; P=8, R=32 (J.X = 8192x8192 @ 8192x256), 200 steps")
SCALING = ["lattice16", "lattice24", "lattice32", "lattice48", "lattice64", "lattice88", "regular1e5", "regular7e5",
           "sk2000", "sk4096", "sk8192", "sk8192t", "skreal2000"]
BYTES_PER_UPDATE = 16  # x, y FP32 read + write per replica-spin update
BYTES_PER_UPDATE_BSB = 20  # ballistic form: + the FP32 f (= x) write
# DRAM traffic per step (dram__bytes_read.sum + dram__bytes_write.sum of one
# ncu capture of the kernel named, divided by the steps of that launch), for
# the roofline's "traffic"; reported only while that kernel is the one that
# runs.  Commands and captures: profiles/*.md.
TRAFFIC_PER_STEP = {
    "regular1e5": {"kernel": "k_solve_csr_persistent", "bytes_per_step": (6372881664 + 7261387008) // 64},
    "lattice16": {"kernel": "k_solve_csr_persistent", "bytes_per_step": (81332736 + 4403397376) // 64},
    "sk2000": {"kernel": "k_solve_dense_tc_f4", "bytes_per_step": (19729664 + 266496) // 1000},
    "lattice16/ballistic": {"kernel": "k_solve_csr_persistent_bsb",
                            "bytes_per_step": (1015867000000 + 999486978000) // 10000},
    "skreal2000": {"kernel": "k_solve_dense_tc_persistent<bf16>", "bytes_per_step": (29336832 + 934400) // 1000},
}
L2_FLUSH_BYTES = 512 << 20
BATCHED_CSR_UPDATES_PER_STEP = 13896704  # the 48-request serving stream's lattice requests


def make_instance(cfg, seed=0):
    if cfg["kind"] == "lattice":
        n, rp, col, val, h = workloads.cubic_lattice(cfg["L"], seed)
        return ("csr", n, rp, col, val, h)
    if cfg["kind"] == "regular":
        n, rp, col, val, h = workloads.random_regular(cfg["n"], cfg["d"], seed, 0.1)
        return ("csr", n, rp, col, val, h)
    if cfg["kind"] == "skreal":
        J, h = workloads.random_dense_real(cfg["n"], seed, 0.1)
        return ("dense", cfg["n"], J, h)
    J, h = workloads.sk_pm1(cfg["n"], seed)
    return ("dense", cfg["n"], J, h)


def n_of(inst):
    return inst[1]


def schedule_params(cfg):
    if cfg["kind"] == "sk" and cfg["n"] == 64:
        return workloads.linear_params(cfg["R"])
    return workloads.autotune_params(cfg["R"], 1)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _loop(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._loop, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for s in self.samples for j in range(4) if len(s) > 4 + j and "Active" in s[4 + j]
                          and "Not" not in s[4 + j]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ------------------------------------------------------------------ reference arm (oracle)
def _oracle_problem(cfg):
    import oracle
    inst = make_instance(cfg)
    if inst[0] == "csr":
        _, n, rp, col, val, h = inst
        pb = oracle.Problem.csr(n, rp, col, val, h)
    else:
        pb = oracle.Problem.dense(inst[2], inst[3])
    return pb.bf16() if cfg["prec"] == "bf16" else pb


def oracle_sample(cfg, target_s=15.0, threads=None):
    """Times the FP64 oracle, as it stands, on a bounded sample of the
    workload (the full instance, all P replicas, a few runs and steps):
    single-threaded for about a third of target_s, then on all host cores
    with one run per thread (runs are independent; the oracle is a C call
    that releases the interpreter lock) for the rest.  The threaded figure is
    the baseline; the single-thread one is reported beside it."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    pb = _oracle_problem(cfg)
    P, S = cfg["P"], cfg["S"]
    variant = 1 if cfg.get("variant") == "ballistic" else 0
    beta, alpha = schedule_params(cfg)
    t0 = time.perf_counter()
    oracle.run(pb, S, P, 1, 0, beta[:1], alpha[:1], n_end=2, variant=variant)
    per_step_run = max((time.perf_counter() - t0) / 2, 1e-6)
    # single thread: a few runs x a few steps, about target_s / 3
    t1 = target_s / 3.0
    runs = max(1, min(cfg["R"], int(t1 / (per_step_run * 100))))
    steps = int(max(2, min(S, t1 / (per_step_run * runs))))
    t0 = time.perf_counter()
    oracle.run(pb, S, P, runs, 0, beta[:runs], alpha[:runs], n_end=steps, variant=variant)
    dt1 = time.perf_counter() - t0
    single = {"value": pb.n * P * runs * steps / dt1, "cores": 1,
              "sample": "%d of %d runs x %d of %d steps, single thread, %.1f s" % (runs, cfg["R"], steps, S, dt1)}
    # all cores: one run per thread, the same number of steps in each
    T = max(1, min(threads or os.cpu_count() or 1, cfg["R"]))
    t2 = target_s - t1
    steps_t = int(max(2, min(S, t2 / per_step_run)))

    def one(r):
        oracle.run(pb, S, P, 1, r, beta[r:r + 1], alpha[r:r + 1], n_end=steps_t, variant=variant)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=T) as ex:
        list(ex.map(one, range(T)))
    dt2 = time.perf_counter() - t0
    return {"value": pb.n * P * T * steps_t / dt2, "unit": "replica-spin updates/s", "cores": T, "kind": "oracle",
            "sample": "%d of %d runs (one per thread) x %d of %d steps, full N=%d and P=%d, %d threads, %.1f s"
                      % (T, cfg["R"], steps_t, S, pb.n, P, T, dt2),
            "single_thread": single}


def run_reference(args, cfg):
    """The reference arm: the oracle as it stands on the host cores.  Each of
    the K timed steps is one bounded sample of the workload (sized so that
    the whole run ends within a couple of minutes); ``ms_per_step`` is the
    measured wall time of one sample, and the time a whole solve would take
    at the sampled rate is reported separately, marked as extrapolated."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    per_sample = max(2.0, min(args.ref_seconds, 90.0 / max(1, args.steps)))
    for _ in range(args.warmup):
        oracle_sample(cfg, target_s=1.0)
    samples, walls = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        samples.append(oracle_sample(cfg, target_s=per_sample))
        walls.append(time.perf_counter() - t0)
    vals = [s["value"] for s in samples]
    value = statistics.mean(vals)
    upd_per_solve = n_of(make_instance(cfg)) * cfg["P"] * cfg["R"] * cfg["S"]
    line = {"impl": "reference", "metric": "replica-spin updates/s", "value": value,
            "unit": "replica-spin updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(walls), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "step_is": "one bounded sample of the workload (ms_per_step = its measured wall time)",
            "extrapolated_ms_per_solve": {"value": 1e3 * upd_per_solve / value, "extrapolated": True,
                                          "note": "a whole solve at the sampled rate; not timed"},
            "config": {"workload": cfg["workload"], "sample": samples[-1]["sample"]},
            "cpu_baseline": dict(samples[-1], value=value),
            "e2e": {"value": value, "unit": "replica-spin updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ serving stream
def batched_csr_roofline(serving, reqs, stream, arena):
    """The engine's CSR chunk kernel alone: a closed loop of the stream's
    lattice requests (no dense work beside it), event-timed launches."""
    lat_reqs = [r for r in reqs if r["inst"]["kind"] == "lattice"]
    csr = serving.run_stream(lat_reqs, None, stream=stream, arena_bytes=arena)
    achieved = BYTES_PER_UPDATE * csr["batched_updates"] / (csr["batched_ms"] * 1e-3) / 1e9
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        peaks = {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    per_step = sum(r["inst"]["n"] * r["P"] * r["R"] for r in lat_reqs)
    # DRAM traffic per step of one ncu capture of this closed loop (the 48-request stream's 19
    # lattice requests, 100-step chunks; profiles/k_solve_batched_serving.md), for that stream only
    traffic = (11023973000 + 12441357000) // 100 if per_step == BATCHED_CSR_UPDATES_PER_STEP else None
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "traffic": traffic, "kernel": "k_solve_batched",
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "algorithmic_bytes_per_step": BYTES_PER_UPDATE * per_step,
            "note": "closed loop of the %d lattice requests alone: algorithmic %d B/update x the updates the "
                    "batched kernel advanced / its event-timed launches" % (len(lat_reqs), BYTES_PER_UPDATE)}


def run_serving_csr(args):
    """`--config serving_csr`: the closed loop of the serving stream's lattice
    requests alone (the engine's CSR chunk kernel), each request of
    --request-steps steps; prints the kernel's roofline record."""
    import torch
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    from paper_2604_01050_gb300 import build as _b
    _b.build()
    from paper_2604_01050_gb300 import serving
    pool = serving.make_pool(12, seed=0)
    reqs = serving.make_requests(pool, args.requests, steps=args.request_steps, R=16, seed=1)
    arena = int(args.arena_gb * (1 << 30))
    lat = [r for r in reqs if r["inst"]["kind"] == "lattice"]
    serving.run_stream(lat[:4], None, stream=stream, arena_bytes=arena)  # warm-up
    roof = batched_csr_roofline(serving, reqs, stream, arena)
    print(json.dumps({"config": {"workload": "closed loop of the lattice requests of the serving stream "
                                             "(%d of %d requests, %d steps each)" % (len(lat), len(reqs),
                                                                                     args.request_steps)},
                      "roofline": roof}))
    for inst in pool:
        inst["problem"].destroy()
    return 0


def plain_serving_compare(serving, pool, reqs, stream, arena, k=8, steps=200):
    """The first k requests of the stream (each cut to `steps` steps) through
    the engine (closed loop) and through the plain per-instance FP32 GPU path
    (torch ops per step, one request after another, readout of the best
    energy per run included), on the same device; replica-spin updates per
    second of each.  The couplings of both sides are resident beforehand."""
    import math
    import torch
    import paper_2604_01050_gb300 as sb
    dev = torch.device("cuda", torch.cuda.current_device())
    sample = [dict(r, steps=steps) for r in reqs[:k]]
    updates = sum(r["inst"]["n"] * r["P"] * r["R"] * steps for r in sample)
    serving.run_stream(sample[:2], None, stream=stream, arena_bytes=arena)  # warm-up
    eng = serving.run_stream(sample, None, stream=stream, arena_bytes=arena)
    mats = {}
    for r in sample:
        q = pool.index(r["inst"])
        if q in mats:
            continue
        pb = r["inst"]["problem"]
        ht = None
        if r["inst"]["kind"] == "sk":
            J, _ = workloads.sk_pm1(r["inst"]["n"], q)
            Jt = torch.tensor(J, dtype=torch.float32, device=dev)
        else:
            L = round(r["inst"]["n"] ** (1.0 / 3.0))
            n, rp, col, val, h = workloads.cubic_lattice(L, q)
            Jt = torch.sparse_csr_tensor(torch.tensor(rp), torch.tensor(col.astype(np.int64)), torch.tensor(val),
                                         size=(n, n), dtype=torch.float32, device=dev)
            ht = None if h is None else torch.tensor(h, dtype=torch.float32, device=dev)
        beta, alpha = workloads.autotune_params(r["R"], q)
        mats[q] = (Jt, ht, beta, alpha, pb.info().c0_auto)

    def plain(r, S):
        Jt, ht, beta, alpha, c0 = mats[pool.index(r["inst"])]
        n, P, R = r["inst"]["n"], r["P"], r["R"]
        ka, dl, kj = schedule_tables(S, P, R, beta, alpha)
        tabs = tuple(torch.tensor(t, dtype=torch.float32, device=dev) for t in (ka, dl, kj))
        g = torch.Generator(device=dev).manual_seed(r["seed"] % (1 << 31))
        x0 = (torch.rand(n, R * P, generator=g, device=dev) - 0.5) * 0.2
        y0 = (torch.rand(n, R * P, generator=g, device=dev) - 0.5) * 0.2
        xf = plain_fp32_solve(Jt, ht, S, P, R, x0, y0, tabs, 0.5 * c0 / P, 0.5 / P, dev)
        spins = torch.where(xf >= 0, 1.0, -1.0)
        e = -0.5 * (spins * (Jt @ spins)).sum(dim=0).double()
        return e.view(R, P).min(dim=1).values.cpu()

    plain(sample[0], 5)  # warm-up (library handles, kernels)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in sample:
        plain(r, steps)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    return {"requests": k, "steps_per_request": steps,
            "engine_updates_per_s": updates / eng["makespan_s"], "engine_s": eng["makespan_s"],
            "plain_fp32_updates_per_s": updates / t_plain, "plain_fp32_s": t_plain,
            "speedup": t_plain / eng["makespan_s"] if eng["makespan_s"] > 0 else math.inf,
            "plain_path": "torch FP32: dense matmul (SK) or CSR SpMM (lattice) per step, then the update, wall and "
                          "threshold as separate elementwise ops; requests one after another"}


def run_serving(args, stream=None):
    """Poisson stream through the batching engine: p50/p99 latency.  Returns
    the JSON record."""
    import torch
    if stream is None:
        torch.cuda.set_device(0)
        stream = torch.cuda.Stream()
    from paper_2604_01050_gb300 import build as _b
    _b.build()
    from paper_2604_01050_gb300 import serving
    pool = serving.make_pool(12, seed=0)
    reqs = serving.make_requests(pool, args.requests, steps=2000, R=16, seed=1)
    arena = int(args.arena_gb * (1 << 30))
    serving.run_stream(reqs[:6], None, stream=stream, arena_bytes=arena)  # warm-up (autotune, first launches)
    closed = serving.run_stream(reqs, None, stream=stream, arena_bytes=arena)
    capacity = len(reqs) / closed["makespan_s"]
    # the same closed loop with every small dense request on its own per-step launches
    unbatched = serving.run_stream(reqs, None, stream=stream, arena_bytes=arena, dense_batching=False)
    loads = {}
    for f in (0.5, 0.8):
        out = serving.run_stream(reqs, f * capacity, stream=stream, seed=int(10 * f), arena_bytes=arena)
        loads["%.1fx" % f] = serving.summary(out)
    # the same stream at fixed request rates, comparable across builds whose capacity differs
    for rate in (30.0, 48.0):
        out = serving.run_stream(reqs, rate, stream=stream, seed=int(rate), arena_bytes=arena)
        loads["%.0f/s" % rate] = serving.summary(out)
    head = loads["0.8x"]
    roof = batched_csr_roofline(serving, reqs, stream, arena)
    vs_plain = plain_serving_compare(serving, pool, reqs, stream, arena)
    cpu = None
    if not args.no_cpu_baseline:
        # the oracle on one typical request (lattice L=16, P=16, R=16, 2000 steps), bounded sample
        cfg = dict(kind="lattice", L=16, P=16, R=16, S=2000, prec="auto")
        base = oracle_sample(cfg, target_s=args.ref_seconds)
        per_req = 16 ** 3 * 16 * 16 * 2000 / base["value"]
        cpu = dict(base, value=per_req, unit="s per request (lattice L=16, P=16, R=16, 2000 steps)")
    line = {"metric": "p99 solve latency", "value": head["p99_s"], "unit": "s", "n_gpus": 1,
            "steps": len(reqs), "warmup": 6, "ms_per_step": 1e3 * head["mean_s"], "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Poisson stream of SK +-1 (dense) and 3D lattice (CSR) requests, "
                                   "N uniform in 64..8192, P in {8,16,32}, R=16, 2000 steps; "
                                   "continuous batching engine, chunk 100 steps",
                       "requests": len(reqs), "arena_gb": args.arena_gb, "capacity_req_per_s": capacity,
                       "closed_loop_updates_per_s": closed["updates"] / closed["makespan_s"],
                       "closed_loop_launches": closed["kernels_launched"],
                       "dense_batched": {"launches": closed["dense_batched_launches"],
                                         "request_chunks": closed["dense_batched_chunks"]},
                       "without_dense_batching": {"capacity_req_per_s": len(reqs) / unbatched["makespan_s"],
                                                  "launches": unbatched["kernels_launched"]}},
            "p50_s": head["p50_s"], "loads": loads, "gpu_launches": head["kernels_launched"],
            "vs_plain_fp32_path": vs_plain,
            "roofline": roof, "cpu_baseline": cpu}
    for inst in pool:
        inst["problem"].destroy()
    return line


# ------------------------------------------------------------------ time-to-epsilon
def plain_fp32_solve(J, h, S, P, R, x0, y0, tables, kc, kx, dev):
    """The plain per-instance FP32 GPU path: per step one library product
    (torch sparse/dense matmul) and separate elementwise kernels, state in
    [N][R*P] FP32 -- the baseline the fused path is compared with."""
    import torch
    x = x0.clone(); y = y0.clone()
    ka, dl, kj = tables
    N = x.shape[0]
    C = R * P
    hcol = torch.zeros(N, 1, device=dev) if h is None else h.view(N, 1)
    kjcols = kj.repeat_interleave(P, dim=1)  # [S][C]
    idx = torch.arange(C, device=dev)
    km = (idx // P) * P + (idx % P + P - 1) % P
    kp = (idx // P) * P + (idx % P + 1) % P
    F = torch.where(x.abs() > dl[0], torch.sign(x), torch.zeros_like(x))
    for n in range(S):
        G = J @ F
        y = y + kc * (G + hcol) - ka[n] * x + kjcols[n] * (x[:, km] + x[:, kp])
        x = x + kx * y
        wall = x.abs() > 1
        x = torch.where(wall, torch.sign(x), x)
        y = torch.where(wall, torch.zeros_like(y), y)
        F = torch.where(x.abs() > dl[n + 1], torch.sign(x), torch.zeros_like(x))
    return x


def schedule_tables(S, P, R, beta, alpha, gamma0=1.0, delta_slope=0.7, a0=1.0, dt=0.5):
    """FP32 step coefficients of the plain path, from the schedule of Sec. II A
    (a(t) = t/T, Gamma_x(t) and J_perp(t) of Eq. 5, Delta(t) of Eq. 8)."""
    tau = np.arange(S + 1) / S
    dl = delta_slope * tau
    ka = dt * (a0 - tau[:S]) / P
    gam = gamma0 * ((1.0 - tau[:S, None]) ** alpha[None, :] + 1e-5)
    jp = -np.log(np.tanh(beta[None, :] * gam / P)) / (2.0 * beta[None, :])
    return ka, dl, dt * jp


def tte_seconds(tau, p, p_target=0.99):
    """Eq. 10; p = 0 gives inf, p >= p_target gives tau."""
    import math
    if p <= 0.0:
        return math.inf
    if p >= p_target:
        return tau
    return tau * math.log(1.0 - p_target) / math.log(1.0 - p)


def run_tte(args):
    """Time-to-epsilon (Eq. 10, p_target = 0.99) of the fused path and of the
    plain FP32 path on the same instance, schedule and initial states."""
    import math
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2604_01050_gb300 import build as _b
    _b.build()
    import paper_2604_01050_gb300 as sb
    L, P, R, S, eps = args.tte_L, 16, 64, args.tte_steps, args.eps
    dense = args.tte_kind == "sk"
    if dense:  # dense SK +-1: the tensor-core path against a dense FP32 matmul per step
        n = args.tte_n
        Jd, hh = workloads.sk_pm1(n, 3)
        prob = sb.create_problem_dense(Jd, hh)
        sum_j2 = float(np.sum(Jd ** 2))
        what = "dense SK N=%d, J=+-1" % n
    else:
        n, rp, col, val, hh = workloads.cubic_lattice(L, 3)
        prob = sb.create_problem_csr(n, rp, col, val, hh)
        sum_j2 = float(np.sum(val ** 2))
        what = "3D cubic lattice L=%d (N=%d), J=+-1" % (L, n)
    beta, alpha = workloads.autotune_params(R, 3)
    sb.set_schedule(prob, beta, alpha, gamma0=args.gamma0)
    # reference energy: best over long, wide searches with the fused path
    E0 = math.inf
    for sd in range(8):
        sb.run(prob, 20 * S, P, R, seed=900 + sd)
        E0 = min(E0, float(sb.get_best(prob)["energy"].min()))
    eps_list = sorted({eps, 0.06, 0.08, 0.10})
    reps = 5
    # fused path: whole solves through the C ABI (init, steps, readout, best to host)
    sb.run(prob, S, P, R, seed=7)
    sb.get_best(prob)
    t0 = time.perf_counter()
    best_f = []
    for k in range(reps):
        sb.run(prob, S, P, R, seed=7 + k)
        best_f.append(sb.get_best(prob)["energy"])
    t_fused = (time.perf_counter() - t0) / reps
    best_f = np.concatenate(best_f)
    # SBM arm: the same runs and kernels with the replica coupling off (J_perp = 0,
    # plain simulated bifurcation per replica), the paper's comparison at equal samples
    sb.set_schedule(prob, beta, alpha, gamma0=args.gamma0, jperp_enable=0)
    sb.run(prob, S, P, R, seed=7)
    sb.get_best(prob)
    best_s = []
    t0 = time.perf_counter()
    for k in range(reps):
        sb.run(prob, S, P, R, seed=7 + k)
        best_s.append(sb.get_best(prob)["energy"])
    t_sb = (time.perf_counter() - t0) / reps
    best_s = np.concatenate(best_s)
    sb.set_schedule(prob, beta, alpha, gamma0=args.gamma0)
    # plain path: same initial states and tables, FP32 torch ops per step
    ka, dl, kj = schedule_tables(S, P, R, beta, alpha, gamma0=args.gamma0)
    c0 = 0.5 * math.sqrt(n / sum_j2)
    kc, kx = 0.5 * c0 / P, 0.5 * 1.0 / P
    tabs = (torch.tensor(ka, dtype=torch.float32, device=dev), torch.tensor(dl, dtype=torch.float32, device=dev),
            torch.tensor(kj, dtype=torch.float32, device=dev))
    if dense:
        Jt = torch.tensor(Jd, dtype=torch.float32, device=dev)
    else:
        Jt = torch.sparse_csr_tensor(torch.tensor(rp), torch.tensor(col.astype(np.int64)), torch.tensor(val),
                                     size=(n, n), dtype=torch.float32, device=dev)
    starts = []
    for k in range(reps):
        sb.run_begin(prob, S, P, R, seed=7 + k)
        x0, y0, _ = sb.get_state(prob)
        starts.append((torch.from_numpy(x0.reshape(R * P, n).T.copy()).to(dev),
                       torch.from_numpy(y0.reshape(R * P, n).T.copy()).to(dev)))
    plain_fp32_solve(Jt, None, 20, P, R, starts[0][0], starts[0][1], tabs, kc, kx, dev)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best_p = []
    for k in range(reps):
        xf = plain_fp32_solve(Jt, None, S, P, R, starts[k][0], starts[k][1], tabs, kc, kx, dev)
        spins = torch.where(xf >= 0, 1.0, -1.0)
        e = -0.5 * (spins * (Jt @ spins)).sum(dim=0).double()
        best_p.append(e.view(R, P).min(dim=1).values.cpu().numpy())
    t_plain = (time.perf_counter() - t0) / reps
    best_p = np.concatenate(best_p)
    E0 = min(E0, float(best_f.min()), float(best_s.min()), float(best_p.min()))
    per_eps = {}
    for e_ in eps_list:
        target = E0 + e_ * abs(E0)
        pf, pp = float(np.mean(best_f <= target)), float(np.mean(best_p <= target))
        ps = float(np.mean(best_s <= target))
        tf, tp, ts = tte_seconds(t_fused / R, pf), tte_seconds(t_plain / R, pp), tte_seconds(t_sb / R, ps)
        per_eps["%g" % e_] = {"p_fused": pf, "p_plain": pp, "tte_fused_s": tf, "tte_plain_s": tp,
                              "speedup": (tp / tf) if math.isfinite(tp) and math.isfinite(tf) else None,
                              "p_sbm": ps, "tte_sbm_s": ts,
                              "sbm_over_sbqa": (ts / tf) if math.isfinite(ts) and math.isfinite(tf) else None}
    head = per_eps["%g" % eps]
    p_fused, p_plain, tte_f, tte_p = head["p_fused"], head["p_plain"], head["tte_fused_s"], head["tte_plain_s"]
    gaps_f = (best_f - E0) / abs(E0)
    line = {"metric": "time-to-epsilon", "value": tte_f, "unit": "s", "n_gpus": 1, "steps": reps, "warmup": 1,
            "ms_per_step": 1e3 * t_fused, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%s, P=%d, R=%d, %d steps, gamma0=%g" % (what, P, R, S, args.gamma0),
                       "epsilon": eps, "E0": E0,
                       "E0_source": "best of 8 x %d runs of %d steps and of every solve timed here" % (R, 20 * S),
                       "p_target": 0.99},
            "fused": {"s_per_solve": t_fused, "p_success": p_fused, "tte_s": tte_f},
            "plain_fp32_torch": {"s_per_solve": t_plain, "p_success": p_plain, "tte_s": tte_p},
            "sbm_jperp0": {"s_per_solve": t_sb, "p_success": head["p_sbm"], "tte_s": head["tte_sbm_s"]},
            "tte_speedup": head["speedup"], "per_epsilon": per_eps,
            "gap_quantiles_fused": [float(np.quantile(gaps_f, q)) for q in (0.0, 0.1, 0.5, 0.9)]}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ (alpha, beta) sensitivity
SWEEP_BETA = [0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 2.0, 3.0, 4.0, 6.0]
SWEEP_ALPHA = [0.25, 0.5, 0.75, 1.0, 1.5, 2.0]


def sweep_layout(alphas, betas, runs, reps):
    """Per-run (beta, alpha) of one batched solve covering the whole grid:
    run index r = ((ia * len(betas) + ib) * runs + q) * reps + t for grid
    point (alphas[ia], betas[ib]), independent run q and repetition t."""
    beta, alpha = [], []
    for a in alphas:
        for b in betas:
            for _ in range(runs * reps):
                beta.append(b)
                alpha.append(a)
    return np.array(beta), np.array(alpha)


def sweep_table(best_energy, alphas, betas, runs, reps, E0):
    """Mean optimality gap (Eq. 9) per grid point: a run's energy is the best
    over its reps repetitions; g is averaged over the runs (the paper's
    sensitivity study, Sec. II B)."""
    e = np.asarray(best_energy, dtype=np.float64).reshape(len(alphas), len(betas), runs, reps).min(axis=3)
    g = (e - E0) / abs(E0)
    return g.mean(axis=2)


def run_sweep(args):
    """Heat maps of the mean optimality gap in the (alpha, beta) plane on
    synthetic instances, with the auto-tuning rule (beta ~ U[0.5, 1.5],
    alpha ~ U[0.5, 1.0] per repetition) beside the grid.  The whole grid of
    one instance is one batched solve (per-run beta, alpha)."""
    import math
    import torch
    torch.cuda.set_device(0)
    from paper_2604_01050_gb300 import build as _b
    _b.build()
    import paper_2604_01050_gb300 as sb
    runs, reps, P = 10, 8, 32
    out = {}
    insts = {"sk512": ("dense SK N=512, J=+-1, h=0", 1000),
             "lattice10": ("3D cubic lattice L=10 (N=1000), J=+-1, h=0", 2000)}
    for name, (desc, S) in insts.items():
        if name.startswith("sk"):
            J, h = workloads.sk_pm1(512, 21)
            prob = sb.create_problem_dense(J, h)
        else:
            n, rp, col, val, hh = workloads.cubic_lattice(10, 21)
            prob = sb.create_problem_csr(n, rp, col, val, hh)
        beta, alpha = sweep_layout(SWEEP_ALPHA, SWEEP_BETA, runs, reps)
        R = len(beta)
        t0 = time.perf_counter()
        sb.set_schedule(prob, beta, alpha, gamma0=args.gamma0)
        sb.run(prob, S, P, R, seed=31)
        grid_best = sb.get_best(prob)["energy"]
        t_grid = time.perf_counter() - t0
        ab, aa = workloads.autotune_params(runs * reps, 32)
        sb.set_schedule(prob, ab, aa, gamma0=args.gamma0)
        sb.run(prob, S, P, runs * reps, seed=32)
        auto_best = sb.get_best(prob)["energy"]
        # control: the same runs with the replica coupling off (plain SB per replica)
        sb.set_schedule(prob, ab, aa, gamma0=args.gamma0, jperp_enable=0)
        sb.run(prob, S, P, runs * reps, seed=32)
        sb_best = sb.get_best(prob)["energy"]
        # reference energy: the best of everything found plus long auto-tuned searches
        E0 = min(float(grid_best.min()), float(auto_best.min()), float(sb_best.min()))
        for sd in range(4):
            sb.run(prob, 10 * S, P, runs * reps, seed=40 + sd)
            E0 = min(E0, float(sb.get_best(prob)["energy"].min()))
        g = sweep_table(grid_best, SWEEP_ALPHA, SWEEP_BETA, runs, reps, E0)
        g_auto = float(((auto_best.reshape(runs, reps).min(axis=1) - E0) / abs(E0)).mean())
        g_sb = float(((sb_best.reshape(runs, reps).min(axis=1) - E0) / abs(E0)).mean())
        gmin = float(g.min())
        ia, ib = np.unravel_index(int(np.argmin(g)), g.shape)
        out[name] = {"instance": desc, "steps": S, "P": P, "runs": runs, "repetitions": reps,
                     "E0": E0, "E0_source": "best over the sweep and 4 x %d auto-tuned runs of %d steps"
                                           % (runs * reps, 10 * S),
                     "alpha": SWEEP_ALPHA, "beta": SWEEP_BETA, "g_mean": [[round(float(v), 5) for v in row] for row in g],
                     "g_min": gmin, "argmin": {"alpha": SWEEP_ALPHA[ia], "beta": SWEEP_BETA[ib]},
                     "within_35pct_of_best": [[bool(v <= 1.35 * gmin) for v in row] for row in g],
                     "g_fixed_alpha1_beta1": float(g[SWEEP_ALPHA.index(1.0), SWEEP_BETA.index(1.0)]),
                     "g_auto_tuned": g_auto, "g_plain_sb_jperp0": g_sb, "grid_solve_s": t_grid,
                     "grid_updates": int(prob.n) * P * R * S}
        prob.destroy()
    print(json.dumps({"metric": "optimality gap g (Eq. 9), mean over runs", "mode": "sweep", "unit": "1",
                      "n_gpus": 1, "gamma0": args.gamma0, "data": "synthetic", "instances": out}))
    return 0


# ------------------------------------------------------------------ large-N scaling
def run_scaling(args):
    """Runs the sparse family one size at a time (each in its own process,
    so device memory is returned between sizes) and prints one line with the
    throughput and roofline fraction of every size: the lattice16 shape from
    an L2-resident state (84 MB) to 14 GB, and the random regular graphs."""
    import subprocess
    points = []
    for name in SCALING:
        cmd = [sys.executable, os.path.abspath(__file__), "--config", name, "--steps", str(args.steps),
               "--warmup", str(args.warmup), "--no-cpu-baseline", "--variant", args.variant]
        out = subprocess.run(cmd, capture_output=True, text=True)
        if out.returncode != 0:
            print(out.stdout[-2000:], out.stderr[-4000:], file=sys.stderr)
            return out.returncode
        line = json.loads(out.stdout.strip().splitlines()[-1])
        c = line["config"]
        points.append({"config": name, "N": c["N"], "P": c["P"], "R": c["R"],
                       "state_MB": round(c["state_bytes"] / 1e6, 1), "value": line["value"],
                       "step_kernel": c["step_kernel"], "step_ms": line["roofline"]["step_ms"],
                       "achieved": line["roofline"]["achieved"], "unit": line["roofline"]["unit"],
                       "bound": line["roofline"]["bound"], "frac": line["roofline"]["frac"],
                       "e2e": line["e2e"]["value"], "clocks": line["clocks"]})
    print(json.dumps({"metric": "replica-spin updates/s", "mode": "scaling", "unit": "replica-spin updates/s",
                      "variant": args.variant, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "points": points}))
    return 0


# ------------------------------------------------------------------ GPU arm
def load_peaks():
    """Measured HBM copy and BF16 GEMM peaks, plus the FP8 e4m3 GEMM
    peak measured by ``bench.py --config fp8peak`` and recorded in
    profiles/fp8_e4m3_dense_peak.md (lines ``fp8_tflops_burst: X``)."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    try:
        for ln in open(os.path.join(ROOT, "profiles", "fp8_e4m3_dense_peak.md")):
            ln = ln.strip().strip("`")
            for key in ("fp8_tflops_burst", "fp8_tflops_sustained", "fp4_tflops_burst", "fp4_tflops_sustained"):
                if ln.startswith(key + ":"):
                    peaks[key] = float(ln.split(":", 1)[1].split()[0])
    except Exception:
        pass
    return peaks


def gpu_context():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2604_01050_gb300 import build as _b
    _b.build()
    import paper_2604_01050_gb300 as sb
    from paper_2604_01050_gb300 import multi
    return {"torch": torch, "sb": sb, "multi": multi, "dist": dist, "rank": rank, "world": world, "dev": dev,
            "stream": torch.cuda.Stream(device=dev), "peaks": load_peaks()}


KERNEL_NAMES = {0: "k_step_csr", 1: "k_step_dense", 2: "k_step_dense_tc", 3: "k_solve_small",
                4: "k_solve_csr_persistent", 5: "k_solve_dense_tc_persistent", 6: "k_step_csr_bsb",
                7: "k_step_dense_bsb", 8: "k_solve_dense_tc_split", 9: "k_solve_dense_tc_pair",
                10: "k_step_dense_tc<bf16>", 11: "k_solve_dense_tc_persistent<bf16>",
                12: "k_step_dense_tc<bsb>", 13: "k_solve_dense_tc_persistent<bsb>", 14: "k_solve_csr_persistent_bsb",
                15: "k_solve_dense_tc_f4", 16: "k_solve_dense_tc_f4_pair"}
KERNEL_LABELS = {0: "csr", 1: "dense_cuda_core", 2: "dense_tcgen05_fp8", 3: "dense_small_one_launch",
                 4: "csr_persistent", 5: "dense_tcgen05_persistent", 6: "csr_ballistic", 7: "dense_ballistic",
                 8: "dense_tcgen05_persistent_split_k", 9: "dense_tcgen05_persistent_cta_pairs",
                 10: "dense_tcgen05_bf16", 11: "dense_tcgen05_persistent_bf16",
                 12: "dense_tcgen05_ballistic_bf16x2", 13: "dense_tcgen05_persistent_ballistic_bf16x2",
                 14: "csr_persistent_ballistic", 15: "dense_tcgen05_persistent_e2m1",
                 16: "dense_tcgen05_persistent_e2m1_cta_pairs"}
TC_FP8 = (2, 5, 8, 9)
TC_BF16 = (10, 11, 12, 13)
TC_FP4 = (15, 16)
FP4_OVER_FP8 = 3.0  # nominal dense e2m1 / e4m3 tensor rate of the GB300 (13.5 / 4.5 PFLOP/s)


def roofline_of(cfg, name, info, N, P, R, step_ms, peaks):
    """The step kernel's roofline: algorithmic bytes (or flops) per step over
    the event-timed step time, against the measured peak of its bound."""
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    kname = KERNEL_NAMES.get(info.step_kernel, "k_%d" % info.step_kernel)
    if info.step_kernel == 2 and (-(-P * R // 128) * 128) % 256 == 0:
        kname = "k_step_dense_tc_wide"  # 128 x 256 tiles when the padded columns allow
    tr = TRAFFIC_PER_STEP.get(name + ("/ballistic" if cfg.get("variant") == "ballistic" else ""))
    traffic = tr["bytes_per_step"] if tr and tr["kernel"] == kname else None
    if info.step_kernel in TC_FP8 + TC_BF16 + TC_FP4:  # a contraction: 2 N^2 R P flops per step
        flops = 2.0 * N * N * P * R
        achieved = flops / (step_ms * 1e-3) / 1e12
        if info.step_kernel in TC_FP4:
            fp8 = peaks.get("fp8_tflops_burst", 2.0 * peaks.get("bf16_tflops", 1900.0))
            if "fp4_tflops_burst" in peaks:
                # a single 8192^3 e2m1 GEMM launch stays below the back-to-back rate: the larger of the two
                peak = max(peaks["fp4_tflops_burst"], peaks.get("fp4_tflops_sustained", 0.0))
                src = "measured (block-scaled e2m1 GEMM, NVFP4 form, profiles/fp8_e4m3_dense_peak.md)"
            else:
                peak = FP4_OVER_FP8 * fp8
                src = "derived: %.0f x measured e4m3 GEMM (profiles/fp8_e4m3_dense_peak.md), nominal e2m1/e4m3 " \
                      "ratio" % FP4_OVER_FP8
            return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic, "kernel": kname, "step_ms": step_ms,
                    "peak_source": src, "frac_of_fp8_peak": achieved / fp8,
                    "note": "2 N^2 R P flops per step / event-timed step time; packed e2m1 operands "
                            "(kind::mxf4), measured dense e2m1 GEMM peak; frac_of_fp8_peak compares with the "
                            "e4m3 solvers"}
        if info.step_kernel in TC_FP8:
            if "fp8_tflops_burst" in peaks:
                peak, src = peaks["fp8_tflops_burst"], "measured (e4m3 GEMM, profiles/fp8_e4m3_dense_peak.md)"
            else:
                peak, src = 2.0 * peaks.get("bf16_tflops", 1900.0), "derived: 2 x measured BF16"
            dt = "FP8 e4m3"
        else:
            peak, src, dt = peaks.get("bf16_tflops", 1900.0), peak_src + " (BF16 GEMM burst)", "BF16"
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "step_ms": step_ms, "peak_source": src,
                "note": "2 N^2 R P flops per step / event-timed step time; %s dense peak" % dt}
    if info.step_kernel == 3:
        # the one-launch small dense solver computes from shared memory and registers: FP32 ALU work,
        # 2 N flops of the product + 12 of the update per replica-spin update, against the FP32 FMA
        # rate of the SMs (152 SMs x 128 lanes x 2 flops x the maximum SM clock)
        flops = (2.0 * N + 12.0) * N * P * R
        achieved = flops / (step_ms * 1e-3) / 1e12
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": kname, "step_ms": step_ms, "peak_source": "derived",
                "note": "(2N + 12) FP32 flops per update / event-timed step time; peak = 152 SMs x 128 FP32 lanes "
                        "x 2 x max SM clock; one CTA per run (%d of 152 SMs busy): latency-bound" % R}
    bpu = BYTES_PER_UPDATE_BSB if info.step_kernel in (6, 7, 14) else BYTES_PER_UPDATE
    achieved_gbs = bpu * N * P * R / (step_ms * 1e-3) / 1e9
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved_gbs / hbm_peak, "traffic": traffic, "kernel": kname, "step_ms": step_ms,
            "peak_source": peak_src, "note": "algorithmic %d B/update x N*P*R per launch / event-timed step time" % bpu}


def measure_config(name, cfg, args, ctx, cpu_seconds):
    """One config: W warm-up solves, K timed solves (CUDA events on the
    library's stream, L2 flushed before each), zero-step solves for the
    step kernel's share, end to end through the C ABI from pinned host
    buffers, and the oracle's bounded CPU sample.  Returns the JSON record."""
    torch, sb, multi, dist = ctx["torch"], ctx["sb"], ctx["multi"], ctx["dist"]
    rank, world, dev, stream, peaks = ctx["rank"], ctx["world"], ctx["dev"], ctx["stream"], ctx["peaks"]
    inst = make_instance(cfg)
    N = n_of(inst)
    P, R, S = cfg["P"], cfg["R"], cfg["S"]
    beta, alpha = schedule_params(cfg)
    upd_per_solve = N * P * R * S
    variant = cfg.get("variant", "threshold")

    def create(src):
        if src[0] == "csr":
            _, n, rp, col, val, h = src
            return sb.create_problem_csr(n, rp, col, val, h)
        return sb.create_problem_dense(src[2], src[3])

    prob = create(inst)
    sb.set_schedule(prob, beta, alpha, precision=cfg["prec"], variant=variant, kernel_select=args.kernel_select)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    seed0 = multi.rank_seed(0, rank)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for w in range(args.warmup):
            sb.run(prob, S, P, R, seed=seed0 + w, stream=stream)
        torch.cuda.synchronize()
        info = prob.info()  # kernel path and autotuner choice of the full solves
        # zero-step solves time init + readout alone (for the step kernel's share)
        sb.run(prob, 0, P, R, seed=seed0, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        ev0 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier()
        with ClockSampler(torch.cuda.current_device()) as clk:
            for k in range(args.steps):
                flush.fill_(float(k))
                ev[k][0].record(stream)
                sb.run(prob, S, P, R, seed=seed0 + 100 + k, stream=stream)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
        barrier()
        for k in range(args.steps):
            flush.fill_(float(k))
            ev0[k][0].record(stream)
            sb.run(prob, 0, P, R, seed=seed0 + k, stream=stream)
            ev0[k][1].record(stream)
        torch.cuda.synchronize()
    prob.destroy()
    del flush
    ms = [a.elapsed_time(b) for a, b in ev]
    ms0 = [a.elapsed_time(b) for a, b in ev0]
    ms_solve = multi.max_over_ranks(statistics.mean(ms))
    ms_zero = statistics.mean(ms0)
    value = world * upd_per_solve / (ms_solve * 1e-3)
    step_ms = max(ms_solve - ms_zero, 1e-9) / S
    roof = roofline_of(cfg, name, info, N, P, R, step_ms, peaks)

    # e2e: host buffers through the C ABI, every step
    src = inst
    if src[0] == "csr":
        _, n, rp, col, val, h = src
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()  # noqa: E731
        src = ("csr", n, pin(rp), pin(col.astype(np.int32)), pin(val), None if h is None else pin(h))
        h2d = (n + 1) * 4 + len(col) * 4 + len(col) * (1 if cfg["prec"] == "auto" else (2 if cfg["prec"] == "bf16" else 4))
        h2d += len(col) * (4 if h is None else 8) + n * (4 + 8)
    else:
        # J as the library uploads it: e4m3 (exact), bfloat16 + the FP64 readout copy (bf16), FP32 + readout copy
        h2d = N * N * {"exact": 1, "bf16": 10}.get(cfg["prec"], 12) + N * (4 + 8)
    h2d += 4 * (2 * S + 1) + 4 * S * R
    d2h = R * N + R * (8 + 8 + 4 + 4)
    e2e_ms = []
    barrier()
    for k in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pe = create(src)
        sb.set_schedule(pe, beta, alpha, precision=cfg["prec"], variant=variant, kernel_select=args.kernel_select)
        sb.run(pe, S, P, R, seed=seed0 + 500 + k, stream=stream)
        best = sb.get_best(pe)
        pe.destroy()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_med_ms = multi.max_over_ranks(statistics.median(e2e_ms))  # the slowest rank
    e2e_val = world * upd_per_solve / (e2e_med_ms * 1e-3)
    assert np.all(np.isfinite(best["energy"]))
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1 and cpu_seconds > 0:
        cpu = oracle_sample(cfg, target_s=cpu_seconds)
    # init + reset_best (+ the f -> e4m3 conversion on the tensor-core path) + steps + 4 readout kernels
    tc_conv = 1 if info.step_kernel in TC_FP8 + TC_BF16 else 0
    persistent = info.step_kernel in (4, 5, 8, 9, 11, 13)
    launches_per_solve = 1 if info.step_kernel == 3 else 2 + tc_conv + (1 if persistent else S) + 4 + tc_conv
    state_b = N * P * R * (18 if variant == "ballistic" else 10)
    return {
        "metric": "replica-spin updates/s", "value": value, "unit": "replica-spin updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_solve,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": cfg["workload"], "name": name, "N": N, "P": P, "R": R, "steps_per_solve": S,
                   "precision": cfg["prec"],
                   "l2": "flushed (512 MB write) before every timed solve; state %.0f MB %s L2 (126 MB) within "
                         "a solve" % (state_b / 1e6, "fits in" if state_b < 100e6 else "exceeds"),
                   "state_bytes": state_b,
                   "parallelism": "independent runs per GPU (weak scaling)",
                   "step_kernel": KERNEL_LABELS.get(info.step_kernel, str(info.step_kernel)),
                   "csr_variant": info.step_variant,
                   "autotune_ms_per_step": [round(v, 5) for v in info.variant_ms],
                   "autotune_persistent_ms_per_step": round(info.persistent_ms, 5)},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "replica-spin updates/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "ms": e2e_med_ms},
        "gpu_launches": launches_per_solve * args.steps,
        "clocks": clk.summary(),
    }


def run_fp8_peak(args):
    """Dense FP8 e4m3 GEMM throughput on this GPU (torch._scaled_mm, unit
    scales, BF16 output, 8192^3): best of 10 single launches (burst) and
    launches back to back for about 4 s (sustained), with the SM clocks
    sampled; a BF16 matmul of the same shape is timed beside it."""
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    n = 8192
    g = torch.Generator(device=dev).manual_seed(0)
    a = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn)
    b = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn).t()  # column-major operand
    one = torch.tensor(1.0, device=dev)
    ab = torch.randn(n, n, device=dev, generator=g, dtype=torch.bfloat16)
    bb = torch.randn(n, n, device=dev, generator=g, dtype=torch.bfloat16)
    fp8 = lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)  # noqa: E731
    bf16 = lambda: ab @ bb  # noqa: E731
    flops = 2.0 * n ** 3
    out = {}
    cases = [("fp8", fp8), ("bf16", bf16)]
    # block-scaled e2m1 GEMM, two values per byte, where this PyTorch has it: NVFP4 form (one e4m3
    # scale per 16 along K; PyTorch 2.9 has no MXFP4 GEMM), every scale 1.0, so the scale tensors'
    # swizzled layout does not matter, only their size
    fp4_note = None
    try:
        a4 = torch.randint(0, 256, (n, n // 2), device=dev, dtype=torch.uint8, generator=g).view(
            torch.float4_e2m1fn_x2)
        b4 = torch.randint(0, 256, (n, n // 2), device=dev, dtype=torch.uint8, generator=g).view(
            torch.float4_e2m1fn_x2)
        sa = torch.full((n, n // 16), 1.0, device=dev).to(torch.float8_e4m3fn)
        sb_ = torch.full((n, n // 16), 1.0, device=dev).to(torch.float8_e4m3fn)
        fp4 = lambda: torch._scaled_mm(a4, b4.t(), scale_a=sa, scale_b=sb_, out_dtype=torch.bfloat16)  # noqa: E731
        fp4()
        torch.cuda.synchronize()
        cases.append(("fp4", fp4))
    except Exception as e:  # no e2m1 GEMM in this PyTorch build
        fp4_note = "%s: %s" % (type(e).__name__, str(e).splitlines()[0][:200] if str(e) else "")
    for name, fn in cases:
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        with ClockSampler(0) as clk:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = max(1, int(4000.0 / best))
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
        out[name] = {"tflops_burst": flops / (best * 1e-3) / 1e12,
                     "tflops_sustained": flops * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12,
                     "sustained_launches": reps, "clocks": clk.summary()}
    print(json.dumps({"metric": "dense GEMM TFLOP/s", "mode": "fp8peak", "shape": [n, n, n],
                      "fp8_e4m3": out["fp8"], "bf16": out["bf16"],
                      "fp4_e2m1_nvfp4": out.get("fp4", {"unavailable": fp4_note}),
                      "fp8_over_bf16_burst": out["fp8"]["tflops_burst"] / out["bf16"]["tflops_burst"],
                      "how": "torch._scaled_mm e4m3 x e4m3 (unit scales, BF16 out), e2m1 x e2m1 (NVFP4 block-16 "
                             "unit scales, BF16 out) and torch.matmul BF16; "
                             "best of 10 (burst), back to back for ~4 s (sustained)"}))
    return 0


HEADLINE = "regular1e5"  # the largest single-GPU configuration (state above L2)
SUBRECORDS = ["lattice16", "sk2000", "skreal2000"]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="default",
                    choices=["default"] + sorted(CONFIGS) + ["serving", "serving_csr", "tte", "scaling", "sweep",
                                                             "fp8peak"],
                    help="default: the random 6-regular N=1e5 headline with per-config records of the lattice "
                         "L=16, dense SK N=2000 and the serving stream; a config name measures that config alone")
    ap.add_argument("--kernel-select", type=int, default=0,
                    help="sbqa_params.kernel_select (0: the autotuner's choice; e.g. 12 pins the 128 x 128 "
                         "persistent dense solver, for profiles)")
    ap.add_argument("--variant", default="threshold", choices=["threshold", "ballistic"],
                    help="f of Eq. 8 (SBQA) or f(x) = x (the bSB form)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="default config: leave out the serving record")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--requests", type=int, default=48, help="serving: requests in the stream")
    ap.add_argument("--arena-gb", type=float, default=40.0, help="serving: device arena of the engine (GB)")
    ap.add_argument("--request-steps", type=int, default=2000, help="serving_csr: steps of each request")
    ap.add_argument("--eps", type=float, default=0.08, help="tte: target optimality gap of the headline")
    ap.add_argument("--gamma0", type=float, default=16.0, help="tte: Gamma_x(0)")
    ap.add_argument("--tte-L", type=int, default=10)
    ap.add_argument("--tte-kind", default="lattice", choices=["lattice", "sk"], help="tte: instance family")
    ap.add_argument("--tte-n", type=int, default=1024, help="tte: N of the dense SK instance")
    ap.add_argument("--tte-steps", type=int, default=2000)
    args = ap.parse_args()
    if args.config == "serving":
        print(json.dumps(run_serving(args)))
        return 0
    if args.config == "serving_csr":
        return run_serving_csr(args)
    if args.config == "tte":
        return run_tte(args)
    if args.config == "scaling":
        return run_scaling(args)
    if args.config == "sweep":
        return run_sweep(args)
    if args.config == "fp8peak":
        return run_fp8_peak(args)
    name = HEADLINE if args.config == "default" else args.config
    cfg = dict(CONFIGS[name])
    if args.variant == "ballistic":
        cfg["variant"] = "ballistic"
        cfg["workload"] += "; ballistic form f(x) = x"
    if args.impl == "reference":
        return run_reference(args, cfg)
    ctx = gpu_context()
    line = measure_config(name, cfg, args, ctx, args.ref_seconds)
    if args.config == "default":
        per = {}
        for sub in SUBRECORDS:
            per[sub] = measure_config(sub, dict(CONFIGS[sub]), args, ctx, min(args.ref_seconds, 10.0))
        if not args.no_serving and ctx["world"] == 1:
            per["serving"] = run_serving(args, stream=ctx["stream"])
        line["per_config"] = per
    if ctx["rank"] == 0:
        print(json.dumps(line))
    if ctx["dist"] is not None:
        ctx["dist"].destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
