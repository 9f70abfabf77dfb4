"""Host-side parts of bench.py (CPU only): the reference arm's JSON line, the
time-to-epsilon formula (Eq. 10) and the schedule tables of the plain FP32
comparison path, checked against the oracle's FP64 schedule."""
import json
import math
import os
import subprocess
import sys

import numpy as np

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` times the oracle on the host and prints one
    JSON line with the contract's keys; its e2e and cpu_baseline values are
    the line's own."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-seconds", "1"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == "replica-spin updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and math.isfinite(d["value"])
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert "workload" in d["config"]
    # a step is one bounded sample: its measured wall time, not a whole solve extrapolated from it
    assert d["ms_per_step"] < 60e3
    assert d["extrapolated_ms_per_solve"]["extrapolated"] is True
    assert d["extrapolated_ms_per_solve"]["value"] > d["ms_per_step"]


def test_tte_seconds_eq10():
    tau = 2.0
    assert bench.tte_seconds(tau, 0.0) == math.inf
    assert bench.tte_seconds(tau, 0.99) == tau and bench.tte_seconds(tau, 1.0) == tau
    # one success in two runs: ln(0.01) / ln(0.5) repetitions
    assert math.isclose(bench.tte_seconds(tau, 0.5), tau * math.log(0.01) / math.log(0.5), rel_tol=1e-15)
    # more successes never cost more time
    ps = np.linspace(0.01, 0.99, 50)
    t = [bench.tte_seconds(tau, p) for p in ps]
    assert all(a >= b for a, b in zip(t, t[1:]))


def test_plain_path_tables_match_the_oracle_schedule():
    """The plain FP32 comparison path builds its step coefficients itself
    (bench.schedule_tables); they must be the oracle's FP64 schedule:
    ka = dt (a0 - a_n) / P, delta_n, dt J_perp(r, n)."""
    S, P, R, dt, gamma0 = 300, 8, 5, 0.5, 16.0
    rng = np.random.default_rng(0)
    beta = rng.uniform(0.5, 1.5, R)
    alpha = rng.uniform(0.5, 1.0, R)
    ka, dl, kj = bench.schedule_tables(S, P, R, beta, alpha, gamma0=gamma0)
    a, d, jp = oracle.schedule(S, P, R, beta, alpha, gamma0, 0.7, True)
    assert np.allclose(ka, dt * (1.0 - a) / P, rtol=1e-14, atol=0)
    assert np.allclose(dl, d, rtol=1e-14, atol=0)
    assert np.allclose(kj, dt * jp.T, rtol=1e-12, atol=0)


class _Info:
    def __init__(self, step_kernel):
        self.step_kernel = step_kernel


def test_roofline_bookkeeping():
    """bench.roofline_of: the dense e2m1 kernels divide 2 N^2 R P flops per step
    by the larger of the measured e2m1 GEMM figures and also report the
    fraction of the e4m3 peak; the ballistic kernels count 20 bytes per
    update, the others 16; a traffic figure is attached only while the kernel
    it was captured on is the one that runs."""
    peaks = {"hbm_gbs": 6633.3, "bf16_tflops": 1908.9, "fp8_tflops_burst": 3587.7, "fp4_tflops_burst": 4687.5,
             "fp4_tflops_sustained": 6949.2}
    N, P, R, ms = 2000, 32, 32, 0.0075
    flops = 2.0 * N * N * P * R
    for k in (15, 16):
        r = bench.roofline_of({}, "sk2000", _Info(k), N, P, R, ms, peaks)
        assert r["bound"] == "tensor" and r["peak"] == 6949.2
        assert math.isclose(r["achieved"], flops / (ms * 1e-3) / 1e12, rel_tol=1e-12)
        assert math.isclose(r["frac_of_fp8_peak"], r["achieved"] / 3587.7, rel_tol=1e-12)
        assert (r["traffic"] is not None) == (bench.KERNEL_NAMES[k] == bench.TRAFFIC_PER_STEP["sk2000"]["kernel"])
    derived = bench.roofline_of({}, "sk2000", _Info(15), N, P, R, ms, {"fp8_tflops_burst": 3587.7})
    assert math.isclose(derived["peak"], bench.FP4_OVER_FP8 * 3587.7, rel_tol=1e-12)
    for k, bpu in ((6, 20), (14, 20), (4, 16), (0, 16)):
        r = bench.roofline_of({}, "lattice16", _Info(k), 4096, 32, 64, 0.0369, peaks)
        assert r["bound"] == "hbm"
        assert math.isclose(r["achieved"], bpu * 4096 * 32 * 64 / (0.0369e-3) / 1e9, rel_tol=1e-12)
    bal = bench.roofline_of({"variant": "ballistic"}, "lattice16", _Info(14), 4096, 32, 64, 0.0369, peaks)
    assert bal["traffic"] == bench.TRAFFIC_PER_STEP["lattice16/ballistic"]["bytes_per_step"]
    thr = bench.roofline_of({}, "lattice16", _Info(6), 4096, 32, 64, 0.0369, peaks)
    assert thr["traffic"] is None  # captured on k_solve_csr_persistent, not the per-step ballistic kernel
