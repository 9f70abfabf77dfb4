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
