"""The BF16 tensor-core product (tcgen05.mma kind::f16, FP32 accumulation in
tensor memory) for dense J that the e4m3 path cannot hold exactly.

Bars (stated once here, used below):
  * real J (precision "bf16"): the product uses J rounded to bfloat16 (round
    to nearest even, the documented quantisation) and f in {-1, 0, +1}, exact
    in bfloat16.  One step from the same FP32 state agrees with the oracle
    on the BF16-rounded J within TOL_STEP = 1e-5 relative, as the CUDA-core
    BF16 path does (only the FP32 summation order differs);
  * integer J with 16 < |J_ij| <= 256 ("exact"): every product and partial sum
    is an exact integer, so the tensor-core state equals the CUDA-core FP32
    state bit for bit, and the readout energies equal the oracle's integers;
  * the ballistic form f(x) = x (Sec. II A, bSB) with "bf16": J rounded to
    bfloat16 and x carried as hi = bf16(x) plus lo = bf16(x - hi), so each
    x_j enters the product with a relative error of at most 2^-16 = 1.5e-5
    (terms of both signs, so G errs far less than that relative to its
    scale); one step from the same state stays within TOL_BSB_STEP = 1e-5 of
    the oracle on the rounded J (measured 2.8e-7), and 100 free-running steps
    within TOL_BSB_TRAJ = 1e-4 (measured 6e-6; f is continuous, so the
    difference grows only through the dynamics);
  * the persistent solver equals the per-step kernel bit for bit (same MMA
    sequence and K order) for all three forms.
"""
import numpy as np
import pytest

import oracle
import workloads
from sbqa_cases import create, dense_int, dense_real, rel_err, wall_ambiguous

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5
TOL_BSB_STEP = 1e-5
TOL_BSB_TRAJ = 1e-4


@pytest.fixture(scope="module")
def sb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as s
    return s


def _params(**kw):
    base = dict(a0=1.0, c0=0.0, dt=0.5, gamma0=1.0, delta_slope=0.7, init_amp=0.1, jperp_enable=1)
    base.update(kw)
    return base


def _per_step(sb, pb, spec, P, R, S, steps, pb_oracle, kernels, seed=3, **pkw):
    prob = create(sb, spec)
    p = _params(**pkw)
    beta, alpha = workloads.autotune_params(R, seed)
    sb.set_schedule(prob, beta, alpha, **p)
    sb.run_begin(prob, S, P, R, seed=seed)
    a, d, jp = oracle.schedule(S, P, R, beta, alpha, p["gamma0"], p["delta_slope"], p["jperp_enable"])
    c0 = p["c0"] if p["c0"] > 0 else oracle.c0_auto(pb)
    kw = dict(a0=p["a0"], c0=c0, dt=p["dt"], variant=1 if p.get("variant") == "ballistic" else 0)
    x, y, _ = sb.get_state(prob)
    worst = 0.0
    for n in range(steps):
        sb.run_advance(prob, 1)
        assert prob.info().step_kernel in kernels, prob.info().step_kernel
        xg, yg, _ = sb.get_state(prob)
        xo = np.empty((R, P, pb.n)); yo = np.empty_like(xo)
        for r in range(R):
            xo[r], yo[r] = oracle.step(pb_oracle, x[r].astype(np.float64), y[r].astype(np.float64), P, a[n], d[n],
                                       jp[r, n], **kw)
        amb = wall_ambiguous(xg, xo)
        worst = max(worst, rel_err(xg, xo), rel_err(np.where(amb, 0.0, yg), np.where(amb, 0.0, yo)))
        x, y = xg, yg
    return worst, prob


@pytest.mark.parametrize("sel,kernel", [(1, 10), (12, 11)])
@pytest.mark.parametrize("N,P,R", [(300, 8, 20), (520, 16, 9)])
def test_bf16_real_dense_per_step_against_oracle(sb, sel, kernel, N, P, R):
    """Real Gaussian J and h: per-step kernel (10) and persistent solver (11), ragged rows and columns."""
    pb, spec = dense_real(N, 5)
    wx, _ = _per_step(sb, pb, spec, P, R, 400, 25, pb.bf16(), (kernel,), precision="bf16", kernel_select=sel,
                      gamma0=4.0 * P)
    print("bf16 tcgen05 per-step worst %.2e (N=%d, P=%d, R=%d, kernel %d)" % (wx, N, P, R, kernel))
    assert wx <= TOL_STEP


@pytest.mark.parametrize("sel", [1, 12])
def test_integer_j_up_to_256_exact_on_bf16_tensor_cores(sb, sel):
    """Integer J with |J| up to 200 (beyond e4m3) and integer h: the BF16 tensor-core product is exact, so
    after 60 steps the state equals the CUDA-core FP32 path bit for bit and the readout energies equal the
    oracle's integers."""
    pb, spec = dense_int(300, 11, jmax=200)
    P, R = 8, 20
    states = []
    for prec in ("exact", "fp32"):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 2), **_params(precision=prec, kernel_select=sel))
        sb.run(prob, 60, P, R, seed=5)
        assert prob.info().step_kernel == ({1: 10, 12: 11}[sel] if prec == "exact" else 1)
        x, y, _ = sb.get_state(prob)
        states.append((x, y))
        e, ei = sb.get_energies(prob)
        assert np.array_equal(ei, oracle.energies(pb, np.where(x >= 0, 1, -1)))
    assert np.array_equal(states[0][0], states[1][0]) and np.array_equal(states[0][1], states[1][1])


@pytest.mark.parametrize("variant", ["threshold", "ballistic"])
def test_bf16_persistent_equals_per_step(sb, variant):
    """The persistent solver and the per-step kernel run the same MMA sequence: bit-identical states after
    45 steps, with readouts every 13 steps, and resume from the middle of the run."""
    pb, spec = dense_real(400, 7)
    P, R = 4, 40
    out = []
    for sel in (1, 12):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 4),
                        **_params(precision="bf16", kernel_select=sel, variant=variant, eval_every=13, gamma0=16.0))
        sb.run_begin(prob, 200, P, R, seed=9)
        sb.run_advance(prob, 20)
        sb.run_advance(prob, 25)
        out.append(sb.get_state(prob)[:2] + (prob.info().step_kernel,))
    base = 10 if variant == "threshold" else 12
    assert out[0][2] == base and out[1][2] == base + 1
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("sel,kernel", [(1, 12), (12, 13)])
def test_ballistic_dense_on_tensor_cores_against_oracle(sb, sel, kernel):
    """bSB (f(x) = x) on the tensor cores: J in bfloat16, x as bfloat16 hi + lo; one step from the same
    state against the oracle's ballistic step on the BF16-rounded J."""
    pb, spec = dense_real(300, 9)
    wx, prob = _per_step(sb, pb, spec, 8, 20, 400, 30, pb.bf16(), (kernel,), precision="bf16", kernel_select=sel,
                         variant="ballistic", gamma0=32.0)
    print("bSB tcgen05 (bf16 hi + lo) per-step worst %.2e (kernel %d)" % (wx, kernel))
    assert wx <= TOL_BSB_STEP


def test_ballistic_dense_tensor_core_free_running_drift(sb):
    """bSB on the tensor cores free-running for 100 steps beside the oracle on the rounded J (Gamma_x(0) =
    4P): the drift is reported and stays within TOL_BSB_TRAJ."""
    pb, spec = dense_real(300, 13)
    P, R, S = 8, 8, 1000
    prob = create(sb, spec)
    beta, alpha = workloads.linear_params(R)
    p = _params(precision="bf16", variant="ballistic", gamma0=32.0)
    sb.set_schedule(prob, beta, alpha, **p)
    sb.run_begin(prob, S, P, R, seed=1)
    ref = oracle.run(pb.bf16(), S, P, R, 1, beta, alpha, gamma0=32.0, n_end=100, n_traj=100,
                     c0=oracle.c0_auto(pb), variant=1)
    errs = []
    for n in range(100):
        sb.run_advance(prob, 1)
        xg, yg, _ = sb.get_state(prob)
        errs.append(max(rel_err(xg, ref["traj_x"][n]), rel_err(yg, ref["traj_y"][n])))
    print("bSB tcgen05 free-running drift at steps 1, 10, 50, 100: %.2e %.2e %.2e %.2e"
          % (errs[0], errs[9], errs[49], errs[99]))
    assert max(errs) <= TOL_BSB_TRAJ


def test_bf16_real_dense_readout_energies(sb):
    """Real J and h on the BF16 tensor-core product: readout energies (FP64 on the CUDA cores, full J) match
    the oracle's energies of the returned spins, and each run's best is its lowest replica."""
    pb, spec = dense_real(384, 3)
    P, R = 16, 16
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, 1), **_params(precision="bf16", gamma0=16.0))
    sb.run(prob, 200, P, R, seed=2)
    assert prob.info().step_kernel in (10, 11)
    e, _ = sb.get_energies(prob)
    x, _, _ = sb.get_state(prob)
    assert np.allclose(e, oracle.energies(pb, np.where(x >= 0, 1, -1)), rtol=1e-12, atol=1e-9)
    best = sb.get_best(prob)
    assert np.array_equal(best["energy"], e.min(axis=1))
