"""Any replica count P (1 <= P <= 128) at the boundary: the Trotter ring of
Eqs. 6-7 (k - 1, k + 1 modulo P, periodic imaginary time) for P that is not
a power of two, and for runs wider than a warp's 32-column chunk (P > 32) on
the tensor cores.

A run of P replicas occupies the next power of two of columns; the columns
past P are padding that no replica reads (the product is per column), so the
kernels differ from the power-of-two case only in where the ring closes.
Bars: the initial state is bit-exact with the oracle's (the random counter
of replica k of run r is (r * P + k) * N + i, as for any P); one step from the
same FP32 state agrees with the oracle within TOL_STEP = 1e-5 relative (the
bar of the other per-step tests); kernels that compute the same exact integer
product (per step, persistent, CUDA cores, tensor cores) agree bit for bit;
readout energies equal the oracle's integers and the best replica of a run
is its lowest one (ties to the lowest k).
"""
import numpy as np
import pytest

import oracle
import workloads
from sbqa_cases import create, dense_int, dense_real, lattice, rel_err, wall_ambiguous

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5


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


def _per_step(sb, pb, spec, P, R, S, steps, kernels, pb_oracle=None, seed=3, **pkw):
    prob = create(sb, spec)
    p = _params(**pkw)
    beta, alpha = workloads.autotune_params(R, seed)
    sb.set_schedule(prob, beta, alpha, **p)
    sb.run_begin(prob, S, P, R, seed=seed)
    a, d, jp = oracle.schedule(S, P, R, beta, alpha, p["gamma0"], p["delta_slope"], p["jperp_enable"])
    c0 = p["c0"] if p["c0"] > 0 else oracle.c0_auto(pb)
    kw = dict(a0=p["a0"], c0=c0, dt=p["dt"], variant=1 if p.get("variant") == "ballistic" else 0)
    x, y, _ = sb.get_state(prob)
    xi, yi = oracle.init_state(seed, pb.n, P, R, 0.1)
    assert np.array_equal(x.astype(np.float64), xi) and np.array_equal(y.astype(np.float64), yi)
    worst = 0.0
    for n in range(steps):
        sb.run_advance(prob, 1)
        assert prob.info().step_kernel in kernels, prob.info().step_kernel
        xg, yg, _ = sb.get_state(prob)
        xo = np.empty((R, P, pb.n)); yo = np.empty_like(xo)
        for r in range(R):
            xo[r], yo[r] = oracle.step(pb_oracle or pb, x[r].astype(np.float64), y[r].astype(np.float64), P, a[n],
                                       d[n], jp[r, n], **kw)
        amb = wall_ambiguous(xg, xo)
        worst = max(worst, rel_err(xg, xo), rel_err(np.where(amb, 0.0, yg), np.where(amb, 0.0, yo)))
        x, y = xg, yg
    return worst, prob


@pytest.mark.parametrize("P,R", [(3, 7), (5, 4), (12, 6), (24, 3), (48, 3), (64, 2), (100, 2), (128, 1)])
def test_csr_per_step_any_p(sb, P, R):
    """3D lattice L=6, CSR per-step kernels (step_kernel 0), ring closing at P."""
    pb, spec = lattice(6, 2)
    w, _ = _per_step(sb, pb, spec, P, R, 300, 20, (0,), kernel_select=1, gamma0=4.0 * P)
    print("CSR P=%d per-step worst %.2e" % (P, w))
    assert w <= TOL_STEP


@pytest.mark.parametrize("P,R", [(3, 50), (12, 20), (48, 8), (64, 6), (100, 4)])
def test_csr_persistent_any_p_equals_per_step(sb, P, R):
    """The persistent CSR solver (step_kernel 4) and the per-step kernels: bit-identical states after 40 steps
    with readouts every 17 steps; and the persistent solver against the oracle for its first steps."""
    pb, spec = lattice(6, 3)
    states = []
    for sel, kern in ((1, 0), (2, 4)):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 5), **_params(kernel_select=sel, eval_every=17,
                                                                           gamma0=4.0 * P))
        sb.run(prob, 40, P, R, seed=11)
        assert prob.info().step_kernel == kern
        states.append(sb.get_state(prob)[:2] + (sb.get_energies(prob)[1], sb.get_best(prob)))
    assert np.array_equal(states[0][0], states[1][0]) and np.array_equal(states[0][1], states[1][1])
    assert np.array_equal(states[0][2], states[1][2])
    w, _ = _per_step(sb, pb, spec, P, R, 300, 8, (4,), kernel_select=2, gamma0=4.0 * P)
    assert w <= TOL_STEP


@pytest.mark.parametrize("P,R", [(3, 40), (12, 11), (48, 3), (64, 4), (100, 3)])
@pytest.mark.parametrize("sel,kern", [(1, 2), (12, 5)])
def test_dense_tensor_cores_any_p(sb, P, R, sel, kern):
    """Integer J on the e4m3 tensor cores, per-step kernel (2) and persistent solver (5), ragged N = 300:
    per-step parity with the oracle, and bit-identical to the CUDA-core FP32 path (an exact product)."""
    pb, spec = dense_int(300, P, jmax=3)
    w, prob = _per_step(sb, pb, spec, P, R, 300, 12, (kern,), precision="exact", kernel_select=sel,
                        gamma0=4.0 * P)
    print("dense tcgen05 P=%d sel %d per-step worst %.2e" % (P, sel, w))
    assert w <= TOL_STEP
    tc_state = sb.get_state(prob)[:2]
    ref = create(sb, spec)
    sb.set_schedule(ref, *workloads.autotune_params(R, 3), **_params(precision="fp32", gamma0=4.0 * P))
    sb.run_begin(ref, 300, P, R, seed=3)
    sb.run_advance(ref, 12)
    assert ref.info().step_kernel == 1
    xr, yr, _ = sb.get_state(ref)
    assert np.array_equal(tc_state[0], xr) and np.array_equal(tc_state[1], yr)


@pytest.mark.parametrize("P", [5, 48])
def test_dense_bf16_tensor_cores_any_p(sb, P):
    """Real J on the BF16 tensor cores (10 per step, 11 persistent) and bSB with x as hi + lo (12, 13)."""
    pb, spec = dense_real(300, 6)
    R = 4
    for sel, kern in ((1, 10), (12, 11)):
        w, _ = _per_step(sb, pb, spec, P, R, 300, 10, (kern,), pb_oracle=pb.bf16(), precision="bf16",
                         kernel_select=sel, gamma0=4.0 * P)
        assert w <= TOL_STEP
    for sel, kern in ((1, 12), (12, 13)):
        w, _ = _per_step(sb, pb, spec, P, R, 300, 10, (kern,), pb_oracle=pb.bf16(), precision="bf16",
                         kernel_select=sel, variant="ballistic", gamma0=4.0 * P)
        assert w <= TOL_STEP


@pytest.mark.parametrize("dense", [False, True])
def test_dense_cuda_core_and_ballistic_any_p(sb, dense):
    """The CUDA-core dense kernel (1) and the ballistic CUDA-core kernels (6, 7) with P = 6 and 40."""
    pb, spec = (dense_real(120, 4) if dense else lattice(5, 4))
    for P in (6, 40):
        w, _ = _per_step(sb, pb, spec, P, 3, 300, 10, (1,) if dense else (0,), precision="fp32", kernel_select=1,
                         gamma0=4.0 * P)
        assert w <= TOL_STEP
        w, _ = _per_step(sb, pb, spec, P, 3, 300, 10, (7,) if dense else (6,), precision="fp32", kernel_select=1,
                         variant="ballistic", gamma0=4.0 * P)
        assert w <= TOL_STEP


@pytest.mark.parametrize("P", [3, 33, 100])
def test_readout_and_best_any_p(sb, P):
    """Energies of all P replicas of every run equal the oracle's integers of the returned spins, the best
    replica is the lowest (ties to the lowest k), and the best spins are that replica's."""
    pb, spec = dense_int(300, 9, jmax=2)
    R = 5
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, 2), **_params(precision="exact", gamma0=16.0))
    sb.run(prob, 120, P, R, seed=4)
    e, ei = sb.get_energies(prob)
    x, _, _ = sb.get_state(prob)
    assert ei.shape == (R, P) and x.shape == (R, P, pb.n)
    spins = np.where(x >= 0, 1, -1).astype(np.int8)
    assert np.array_equal(ei, oracle.energies(pb, spins))
    best = sb.get_best(prob)
    for r in range(R):
        k = int(np.argmin(ei[r]))
        assert best["replica"][r] == k and best["energy"][r] == ei[r, k]
        assert np.array_equal(best["spins"][r], spins[r, k])


def test_set_state_any_p_resume(sb):
    """Checkpoint / resume with P = 7: set_state of a mid-run state continues bit for bit."""
    pb, spec = lattice(5, 1)
    P, R = 7, 5
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, 1), **_params(gamma0=28.0))
    sb.run_begin(prob, 200, P, R, seed=8)
    sb.run_advance(prob, 30)
    xm, ym, sd = sb.get_state(prob)
    sb.run_advance(prob, 30)
    xa, ya, _ = sb.get_state(prob)
    sb.set_state(prob, xm, ym, sd)
    sb.run_advance(prob, 30)
    xb, yb, _ = sb.get_state(prob)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


def test_engine_any_p_mix_equals_alone(sb):
    """The batching engine serves P = 3, 12 and 48 (CSR batched kernel, dense tensor cores) bit for bit
    as sbqa_run does."""
    reqs = []
    for k, (spec, P, R) in enumerate([(lattice(6, 1)[1], 3, 6), (lattice(5, 2)[1], 12, 4), (lattice(6, 3)[1], 48, 2),
                                      (dense_int(300, 4, jmax=2)[1], 12, 4), (dense_int(280, 5, jmax=2)[1], 48, 2)]):
        pb = create(sb, spec)
        sb.set_schedule(pb, *workloads.autotune_params(R, k), precision="exact" if spec[0] == "dense" else "auto",
                        gamma0=4.0 * P)
        reqs.append((pb, 60, P, R, 200 + k))
    alone = []
    for pb, steps, P, R, seed in reqs:
        sb.run(pb, steps, P, R, seed=seed)
        alone.append(sb.get_best(pb))
    eng = sb.engine_create(256 << 20, 8, 16)
    ids = [sb.engine_submit(eng, *r) for r in reqs]
    done = []
    for _ in range(1000):
        done += sb.engine_step(eng)
        if len(done) == len(ids):
            break
    assert sorted(done) == ids
    for rid, ref in zip(ids, alone):
        got = sb.engine_result(eng, rid)
        assert np.array_equal(got["energy"], ref["energy"]) and np.array_equal(got["spins"], ref["spins"])
        assert np.array_equal(got["replica"], ref["replica"])
