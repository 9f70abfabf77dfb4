"""Parity of the CUDA hot path (through the C ABI) with the FP64 oracle.

Bars (stated once here, used below):
  * initial state: bit-exact (both sides implement SplitMix64);
  * one step from the same FP32 state: relative error <= 1e-5 per (run,
    replica) for x and y (TOL_STEP); elements where the strict wall test
    |x| > 1 falls on different sides in FP32 and FP64 are listed and excluded
    from the y comparison (their x agree to 4e-6);
  * free-running FP32 trajectories vs the FP64 oracle: <= 1e-5 relative per
    step (TOL_TRAJ) for 100 steps at Gamma_x(0) = 4P (theta = beta Gamma/P = 4
    keeps J_perp below the restoring force (a0 - a)/(2P), so the in-phase
    replica mode is stable), and for the first 20 steps at Gamma_x(0) = 1,
    where that mode is linearly unstable from t = 0 and amplifies rounding
    differences;
  * the threshold f of Eq. 8 is decided in FP32 by the kernels and in FP64 by
    the oracle: positions within 1e-6 of Delta are counted as
    threshold-sensitive, and every position where the two decisions differ
    is listed by seed and step (never excluded from a comparison);
  * integer energies: bit-exact; real energies: 1e-12 relative (FP64 sums in
    another order);
  * BF16 product: against the oracle on the BF16-rounded J, TOL_STEP per step
    and 1e-4 (TOL_BF16_TRAJ) for 100 free-running steps (real J and h: the
    FP32 sums of rounded products drift a little faster than the exact
    integer sums); against the unrounded J, one step from the same
    state stays within 1e-2 relative (TOL_BF16_STEP; the quantisation of J to
    8 significant bits gives about 1e-3).  Free-running trajectories on the
    two J's separate after a few steps because the rounding moves x across
    the threshold Delta (f is discontinuous), so no multi-step bound against
    the unrounded J is claimed;
  * best-energy distributions over 256 runs: permutation test on the mean
    and chi-square over integer energy bins, both p > 0.01.
"""
import numpy as np
import pytest

import oracle
import workloads
from sbqa_cases import create, dense_int, dense_real, lattice, regular, rel_err, sk, wall_ambiguous

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-5
TOL_TRAJ = 1e-5
TOL_BF16_STEP = 1e-2
TOL_BF16_TRAJ = 1e-4


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


def _oracle_kwargs(p, pb):
    c0 = p["c0"] if p["c0"] > 0 else oracle.c0_auto(pb)
    return dict(a0=p["a0"], c0=c0, dt=p["dt"], variant=p.get("variant", 0))


# ---------------------------------------------------------------- initial state
@pytest.mark.parametrize("N,P,R", [(64, 8, 16), (33, 2, 3), (7, 1, 5), (130, 32, 5), (1, 4, 2)])
def test_initial_state_bit_exact(sb, N, P, R):
    pb, spec = sk(N, 1) if N > 1 else (oracle.Problem.dense(np.zeros((1, 1))), ("dense", np.zeros((1, 1)), None))
    prob = create(sb, spec)
    beta, alpha = workloads.autotune_params(R, 0)
    sb.set_schedule(prob, beta, alpha, **_params())
    sb.run_begin(prob, 10, P, R, seed=12345)
    xg, yg, sd = sb.get_state(prob)
    xo, yo = oracle.init_state(12345, N, P, R, 0.1)
    assert sd == 0
    assert np.array_equal(xg.astype(np.float64), xo) and np.array_equal(yg.astype(np.float64), yo)


# ---------------------------------------------------------------- one step from the same state
def _per_step(sb, pb, spec, P, R, S, steps, seed=3, prec="auto", pb_oracle=None, **pkw):
    prob = create(sb, spec)
    p = _params(precision=prec, **pkw)
    beta, alpha = workloads.autotune_params(R, seed)
    sb.set_schedule(prob, beta, alpha, **p)
    sb.run_begin(prob, S, P, R, seed=seed)
    ref = pb_oracle or pb
    a, d, jp = oracle.schedule(S, P, R, beta, alpha, p["gamma0"], p["delta_slope"], p["jperp_enable"])
    kw = _oracle_kwargs(p, pb)
    x, y, _ = sb.get_state(prob)
    worst_x = worst_y = 0.0
    amb_total = 0
    thr_total, thr_steps = 0, []
    flips = []
    for n in range(steps):
        # threshold-sensitive: a position within 1e-6 of the threshold that decides f(x_n) (Eq. 8),
        # where FP32 and FP64 may take different sides; reported, never excluded
        near = int((np.abs(np.abs(x.astype(np.float64)) - d[n]) < 1e-6).sum())
        if near:
            thr_total += near
            thr_steps.append(n)
        nf = _threshold_flips(x, x.astype(np.float64), d[n])
        if nf:
            flips.append((n, nf))
        sb.run_advance(prob, 1)
        xg, yg, sd = sb.get_state(prob)
        assert sd == n + 1
        xo = np.empty((R, P, pb.n)); yo = np.empty_like(xo)
        for r in range(R):
            xo[r], yo[r] = oracle.step(ref, x[r].astype(np.float64), y[r].astype(np.float64), P, a[n], d[n],
                                       jp[r, n], **kw)
        amb = wall_ambiguous(xg, xo)
        amb_total += int(amb.sum())
        worst_x = max(worst_x, rel_err(xg, xo))
        yg_c = np.where(amb, 0.0, yg); yo_c = np.where(amb, 0.0, yo)
        worst_y = max(worst_y, rel_err(yg_c, yo_c))
        x, y = xg, yg
    if thr_total:
        print("threshold-sensitive positions: %d at steps %s (seed %d)" % (thr_total, thr_steps[:20], seed))
    if flips:
        print("FP32/FP64 threshold flips (step, count): %s (seed %d)" % (flips[:20], seed))
    return worst_x, worst_y, amb_total, prob


def _threshold_flips(x32, x64, delta):
    """Positions whose f of Eq. 8 differs between the kernel's decision (|x| <= Delta compared in
    FP32, on its FP32 state and the FP32-rounded Delta) and the oracle's (FP64 state, FP64 Delta)."""
    dev = np.abs(np.asarray(x32, dtype=np.float32)) <= np.float32(delta)
    orc = np.abs(np.asarray(x64, dtype=np.float64)) <= delta
    return int((dev != orc).sum())


def test_per_step_dense_sk64_default_schedule(sb):
    """Config-1 shape: dense SK N=64 +-1, P=8, R=16, 1000-step schedule; every one of the first 100 steps."""
    pb, spec = sk(64, 0)
    wx, wy, amb, _ = _per_step(sb, pb, spec, 8, 16, 1000, 100)
    print("per-step worst x %.2e y %.2e wall-ambiguous %d" % (wx, wy, amb))
    assert wx <= TOL_STEP and wy <= TOL_STEP


def test_per_step_lattice_csr(sb):
    pb, spec = lattice(6, 2)
    wx, wy, amb, _ = _per_step(sb, pb, spec, 32, 4, 500, 60)
    assert wx <= TOL_STEP and wy <= TOL_STEP


@pytest.mark.parametrize("P,R", [(1, 5), (2, 3), (4, 7), (16, 3)])
def test_per_step_ragged_shapes(sb, P, R):
    pb, spec = lattice(3, 5)  # N = 27: a ragged tail of rows
    wx, wy, _, _ = _per_step(sb, pb, spec, P, R, 200, 30, seed=P)
    assert wx <= TOL_STEP and wy <= TOL_STEP


def test_per_step_real_sparse_fp32_with_field(sb):
    pb, spec = regular(500, 6, 1)
    wx, wy, _, _ = _per_step(sb, pb, spec, 16, 8, 300, 40, prec="fp32")
    assert wx <= TOL_STEP and wy <= TOL_STEP


def test_per_step_real_sparse_bf16(sb):
    """BF16 product: parity against the oracle on the BF16-rounded J."""
    pb, spec = regular(500, 6, 2)
    wx, wy, _, _ = _per_step(sb, pb, spec, 16, 8, 300, 40, prec="bf16", pb_oracle=pb.bf16())
    assert wx <= TOL_STEP and wy <= TOL_STEP


def test_per_step_dense_real_and_integer(sb):
    pb, spec = dense_real(100, 3)
    wx, wy, _, _ = _per_step(sb, pb, spec, 8, 4, 200, 30, prec="fp32")
    assert wx <= TOL_STEP and wy <= TOL_STEP
    pb, spec = dense_int(90, 4)
    wx, wy, _, _ = _per_step(sb, pb, spec, 4, 4, 200, 30, prec="exact")
    assert wx <= TOL_STEP and wy <= TOL_STEP


def test_per_step_jperp_disabled(sb):
    pb, spec = sk(48, 6)
    wx, wy, _, _ = _per_step(sb, pb, spec, 8, 4, 200, 30, jperp_enable=0)
    assert wx <= TOL_STEP and wy <= TOL_STEP


@pytest.mark.parametrize("sel", [1, 2])
@pytest.mark.parametrize("jmax,P,R", [(1, 8, 5), (3, 32, 4), (16, 2, 7), (16, 16, 9)])
def test_dense_tensor_core_path_bit_exact_with_cuda_cores(sb, jmax, P, R, sel):
    """Integer J on the tcgen05 FP8 path (N >= 256; per-step kernel for sel=1,
    the persistent solver for sel=2) and on the CUDA-core FP32 path compute
    the same exact product and the same update: states agree bit for bit
    after 60 steps (ragged rows N = 300, ragged columns R * P)."""
    pb, spec = dense_int(300, jmax, jmax=jmax)
    states = []
    for prec in ("exact", "fp32"):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 2), **_params(precision=prec, kernel_select=sel))
        sb.run_begin(prob, 400, P, R, seed=5)
        sb.run_advance(prob, 60)
        assert prob.info().step_kernel == ({1: 2, 2: 5}[sel] if prec == "exact" else 1)
        states.append(sb.get_state(prob)[:2])
    assert np.array_equal(states[0][0], states[1][0]) and np.array_equal(states[0][1], states[1][1])


def _split_k(N, P, R):
    """The persistent tcgen05 solver splits its K loop across 2-CTA clusters
    when padded N and padded R * P are multiples of 256."""
    pad = lambda v: -(-v // 128) * 128
    return pad(N) % 256 == 0 and pad(P * R) % 256 == 0


def _pair(N):
    """The paired persistent solver (2-CTA clusters sharing M=256 MMAs) takes
    padded N a multiple of 256."""
    return -(-N // 128) * 128 % 256 == 0


@pytest.mark.parametrize("N,P,R,jmax", [(300, 8, 40, 3), (512, 16, 16, 1), (1000, 32, 32, 1), (260, 4, 33, 16),
                                        (500, 8, 48, 5), (700, 2, 128, 1), (1000, 16, 9, 2)])
def test_persistent_dense_tc_solver_matches_per_step(sb, N, P, R, jmax):
    """The persistent tcgen05 solvers (x, y resident in tensor memory, per-tile
    step flags between CTAs; 128 x 128 tiles; where padded N and R * P are
    multiples of 256 the split-K solver on 2-CTA clusters; where padded N is
    a multiple of 256 the paired solver whose 2-CTA clusters share M=256
    MMAs; with |J_ij| <= 4 the solver with packed e2m1 operands) and the
    per-step tcgen05 kernel give bit-identical runs, readouts
    every 37 steps included; ragged row and column tiles (N = 300, 260, 500,
    700, 1000; R * P = 320, 132, 384, 144)."""
    pb, spec = dense_int(N, N + R, jmax=jmax)
    out = []
    for sel in (1, 2, 12, 13, 14):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, N), **_params(kernel_select=sel, eval_every=37))
        sb.run(prob, 200, P, R, seed=N)
        want = {1: 2, 2: 8 if _split_k(N, P, R) else 5, 12: 5, 13: 9 if _pair(N) else 5,
                14: (16 if _pair(N) else 15) if jmax <= 4 else 5}[sel]
        assert prob.info().step_kernel == want
        out.append((sb.get_state(prob)[:2], sb.get_energies(prob), sb.get_best(prob)))
    (xa, ya), ea, ba = out[0]
    for (xb, yb), eb, bb in out[1:]:
        assert np.array_equal(xa, xb) and np.array_equal(ya, yb)
        assert np.array_equal(ea[1], eb[1])
        for k in ba:
            assert np.array_equal(ba[k], bb[k]), k
    _check_best_with_readouts(sb, pb, prob, R, 200, 37)


@pytest.mark.parametrize("N,P,R,jmax", [(300, 8, 5, 3), (700, 16, 24, 16), (260, 32, 4, 1)])
def test_dense_tensor_core_readout_matches_cuda_cores(sb, N, P, R, jmax):
    """Readout energies of integer dense instances on the tensor cores (sign
    codes through one FP8 GEMM, exact integer row sums in its epilogue) equal
    the CUDA-core readout and the oracle's energies of the final spins, and
    the best-so-far over readouts every 29 steps agrees (ragged N and R * P,
    integer h)."""
    pb, spec = dense_int(N, N + 7, jmax=jmax)
    res = []
    for prec in ("exact", "fp32"):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 5), **_params(precision=prec, eval_every=29))
        sb.run(prob, 120, P, R, seed=7)
        assert (prob.info().step_kernel in (2, 5, 8, 9, 15, 16)) if prec == "exact" else prob.info().step_kernel == 1
        _, ei = sb.get_energies(prob)
        x, _, _ = sb.get_state(prob)
        res.append((ei, sb.get_best(prob), x))
    (ea, ba, xa), (eb, bb, xb) = res
    assert np.array_equal(xa, xb)
    assert np.array_equal(ea, eb)
    for k in ba:
        assert np.array_equal(ba[k], bb[k]), k
    assert np.array_equal(ea, oracle.energies(pb, np.where(xa >= 0, 1, -1)))


def test_cached_device_blocks_give_identical_runs(sb):
    """Handles created after others were destroyed take their device buffers
    from the library's cache, old contents included; their runs equal the
    first handle's bit for bit, and so do runs after the cache was returned to
    the driver (dense on the tensor cores, and a +-1 lattice in CSR)."""
    for spec, P, R in ((sk(384, 3)[1], 16, 8), (lattice(6, 2)[1], 8, 16)):
        res = []
        for k in range(4):
            prob = create(sb, spec)
            sb.set_schedule(prob, *workloads.autotune_params(R, 2), **_params(eval_every=23))
            sb.run(prob, 90, P, R, seed=11)
            res.append((sb.get_state(prob)[:2], sb.get_energies(prob)[1], sb.get_best(prob)))
            prob.destroy()
            if k == 2:
                sb.release_cached_memory()
        (xa, ya), ea, ba = res[0]
        for (xb, yb), eb, bb in res[1:]:
            assert np.array_equal(xa, xb) and np.array_equal(ya, yb) and np.array_equal(ea, eb)
            for key in ba:
                assert np.array_equal(ba[key], bb[key]), key


@pytest.mark.parametrize("jmax,real_h", [(100, False), (100, True), (200, False), (16, True)])
def test_dense_host_copy_forms(sb, jmax, real_h):
    """The library keeps a dense integer J with |J_ij| <= 127 as one byte per
    entry and any other J in FP64: the readout energies of the final spins
    equal the oracle's (exact for integer J and h, 1e-12 relative with a real
    h), with the FP32 step path and the tensor-core path alike."""
    N, P, R = 300, 4, 6
    rng = np.random.default_rng(jmax + real_h)
    up = np.triu(rng.integers(-jmax, jmax + 1, (N, N)).astype(float), 1)
    J = up + up.T
    h = rng.normal(0.0, 0.7, N) if real_h else rng.integers(-3, 4, N).astype(float)
    pb = oracle.Problem.dense(J, h)
    for prec in (("exact", "fp32") if jmax <= 256 else ("fp32",)):  # exact: e4m3 up to 16, bf16 tensor cores above
        prob = sb.create_problem_dense(J, h)
        sb.set_schedule(prob, *workloads.autotune_params(R, 4), **_params(precision=prec))
        sb.run(prob, 60, P, R, seed=5)
        x, _, _ = sb.get_state(prob)
        e, ei = sb.get_energies(prob)
        ref = oracle.energies(pb, np.where(x >= 0, 1, -1))
        if real_h:
            assert np.allclose(e, ref, rtol=1e-12, atol=1e-9)
        else:
            assert np.array_equal(ei, ref)
        prob.destroy()


@pytest.mark.parametrize("N,sel,want", [(384, 2, 5), (512, 2, 8), (768, 13, 9)])
def test_persistent_dense_tc_solver_resume(sb, N, sel, want):
    """Stretches of the persistent tcgen05 solvers (128 x 128 tiles at N =
    384; split-K clusters at N = 512; CTA pairs at N = 768) resumed across
    begin/advance/finish give the state of one uninterrupted run."""
    pb, spec = sk(N, 9)
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(16, 9), **_params(kernel_select=sel))
    sb.run(prob, 150, 16, 16, seed=4)
    xa, ya, _ = sb.get_state(prob)
    sb.run_begin(prob, 150, 16, 16, seed=4)
    sb.run_advance(prob, 1)
    sb.run_advance(prob, 60)
    sb.run_advance(prob, 500)
    sb.run_finish(prob)
    xb, yb, _ = sb.get_state(prob)
    assert prob.info().step_kernel == want
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


@pytest.mark.parametrize("N,P,R", [(384, 32, 4), (300, 16, 12), (520, 32, 16)])
def test_per_step_dense_tensor_core_sk(sb, N, P, R):
    """Per-step tcgen05 kernels against the oracle step by step: 128-column
    tiles (R * P = 128) and 256-column tiles (R * P = 192 in a padded 256,
    ragged; 512 in two tiles), ragged spin rows (N = 300, 520)."""
    pb, spec = sk(N, 3)
    wx, wy, _, _ = _per_step(sb, pb, spec, P, R, 1000, 40, prec="exact")
    assert wx <= TOL_STEP and wy <= TOL_STEP


# ---------------------------------------------------------------- free-running trajectories
def _free_running(sb, pb, spec, P, R, S, steps, gamma0, seed=0, prec="auto", pb_oracle=None, **pkw):
    prob = create(sb, spec)
    p = _params(gamma0=gamma0, precision=prec, **pkw)
    beta, alpha = workloads.linear_params(R)
    sb.set_schedule(prob, beta, alpha, **p)
    sb.run_begin(prob, S, P, R, seed=seed)
    ref = oracle.run(pb_oracle or pb, S, P, R, seed, beta, alpha, gamma0=gamma0, n_end=steps, n_traj=steps,
                     **_oracle_kwargs(p, pb))
    a, d, _ = oracle.schedule(S, P, R, beta, alpha, gamma0)
    errs = []
    flips = []
    for n in range(steps):
        sb.run_advance(prob, 1)
        xg, yg, _ = sb.get_state(prob)
        errs.append((rel_err(xg, ref["traj_x"][n]), rel_err(yg, ref["traj_y"][n])))
        # the decision of f (Eq. 8) that the next step takes, on each side's own state
        nf = _threshold_flips(xg, ref["traj_x"][n], d[n + 1]) if n + 1 < steps else 0
        if nf:
            flips.append((n + 1, nf, float(errs[-1][0])))
    if flips:
        print("FP32/FP64 threshold flips (step, count, x error before it): %s (seed %d)" % (flips[:20], seed))
    return np.array(errs)


def test_free_running_sk64_100_steps_stable_schedule(sb):
    pb, spec = sk(64, 0)
    e = _free_running(sb, pb, spec, 8, 16, 1000, 100, gamma0=32.0)
    print("free-running max x %.2e y %.2e" % tuple(e.max(axis=0)))
    assert e.max() <= TOL_TRAJ


def test_free_running_sk64_default_schedule_first_20_steps(sb):
    pb, spec = sk(64, 0)
    e = _free_running(sb, pb, spec, 8, 16, 1000, 40, gamma0=1.0)
    print("gamma0=1 divergence by step:", ["%.1e" % v for v in e.max(axis=1)[::5]])
    assert e[:20].max() <= TOL_TRAJ


def test_free_running_lattice_100_steps(sb):
    pb, spec = lattice(8, 1)
    e = _free_running(sb, pb, spec, 32, 4, 1000, 100, gamma0=128.0)
    assert e.max() <= TOL_TRAJ


def test_bf16_against_unrounded_j(sb):
    pb, spec = regular(400, 6, 7)
    wx, wy, _, _ = _per_step(sb, pb, spec, 16, 4, 1000, 60, prec="bf16", gamma0=64.0)
    print("bf16 per-step error vs FP64 J: x %.2e y %.2e" % (wx, wy))
    assert wx <= TOL_BF16_STEP and wy <= TOL_BF16_STEP
    e = _free_running(sb, pb, spec, 16, 4, 1000, 100, gamma0=64.0, prec="bf16", pb_oracle=pb.bf16())
    print("bf16 free-running vs oracle on the rounded J: %.2e" % e.max())
    assert e.max() <= TOL_BF16_TRAJ


# ---------------------------------------------------------------- energies and best
def _check_energies_and_best(sb, pb, prob, R, P):
    e, ei = sb.get_energies(prob)
    x, _, _ = sb.get_state(prob)
    spins = np.where(x >= 0, 1, -1).astype(np.int8)
    ref = oracle.energies(pb, spins)
    if pb.is_integer:
        assert np.array_equal(ei, ref) and np.array_equal(e, ref.astype(float))
    else:
        assert np.allclose(e, ref, rtol=1e-12, atol=1e-9)
    best = sb.get_best(prob)
    for r in range(R):
        k = int(np.argmin(e[r]))
        assert best["replica"][r] == k
        assert best["energy"][r] == e[r, k]
        assert np.array_equal(best["spins"][r], spins[r, k])
        eb = oracle.energy_int(pb, best["spins"][r]) if pb.is_integer else oracle.energy(pb, best["spins"][r])
        assert eb == pytest.approx(best["energy"][r], rel=1e-12, abs=1e-9)
    return best


def test_full_run_dense_tensor_core_energies_exact(sb):
    pb, spec = sk(512, 4)
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(8, 4), **_params(precision="exact"))
    sb.run(prob, 300, 16, 8, seed=3)
    _check_energies_and_best(sb, pb, prob, 8, 16)


@pytest.mark.parametrize("N,P,R,S,jmax", [(64, 8, 16, 300, 1), (100, 4, 5, 150, 3), (48, 1, 7, 100, 2),
                                         (128, 8, 3, 200, 1), (33, 16, 2, 80, 4)])
def test_small_one_launch_solver_matches_per_step_path(sb, N, P, R, S, jmax):
    """Small integer dense instances solve in one launch; state, energies and
    best agree bit for bit with the per-step kernels (begin/advance/finish)."""
    pb, spec = dense_int(N, N + P, jmax=jmax)
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, N), **_params())
    sb.run(prob, S, P, R, seed=N)
    assert prob.info().step_kernel == 3
    xa, ya, _ = sb.get_state(prob)
    ea = sb.get_energies(prob)
    ba = sb.get_best(prob)
    sb.run_begin(prob, S, P, R, seed=N)
    sb.run_advance(prob, S)
    sb.run_finish(prob)
    assert prob.info().step_kernel == 1
    xb, yb, _ = sb.get_state(prob)
    eb = sb.get_energies(prob)
    bb = sb.get_best(prob)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)
    assert np.array_equal(ea[0], eb[0]) and np.array_equal(ea[1], eb[1])
    for k in ba:
        assert np.array_equal(ba[k], bb[k]), k
    _check_energies_and_best(sb, pb, prob, R, P)


@pytest.mark.parametrize("case", ["lattice", "regular_f32", "regular_bf16", "ragged", "degree12"])
def test_csr_step_variants_bit_identical(sb, case):
    """Every per-step CSR kernel variant (W = 4, 8, 16 columns per lane; one
    item per warp or one wave of blocks looping over the items; the ELL form
    for degree <= 8, which falls back to variant 0 at degree 12), forced with
    kernel_select = 3 + v, gives the same state bit for bit after 40 steps."""
    if case == "lattice":
        pb, spec = lattice(8, 1); P, R, prec = 32, 16, "auto"
    elif case == "regular_f32":
        pb, spec = regular(700, 6, 3); P, R, prec = 16, 32, "fp32"
    elif case == "regular_bf16":
        pb, spec = regular(700, 5, 4); P, R, prec = 8, 64, "bf16"
    elif case == "ragged":
        pb, spec = lattice(5, 2); P, R, prec = 32, 5, "auto"  # Cp = 256: W = 16 falls back
    else:
        pb, spec = regular(400, 12, 5); P, R, prec = 16, 16, "fp32"
    states = []
    for v in range(8):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 3), **_params(precision=prec, kernel_select=3 + v))
        sb.run_begin(prob, 300, P, R, seed=11)
        sb.run_advance(prob, 40)
        info = prob.info()
        assert info.step_kernel == 0
        states.append(sb.get_state(prob)[:2])
    for v in range(1, 8):
        assert np.array_equal(states[0][0], states[v][0]) and np.array_equal(states[0][1], states[v][1]), v


@pytest.mark.parametrize("variant", [3, 6])
def test_csr_grid_stride_and_ell_variants_against_oracle(sb, variant):
    pb, spec = regular(500, 6, 1)
    wx, wy, _, prob = _per_step(sb, pb, spec, 16, 8, 300, 30, prec="fp32", kernel_select=3 + variant)
    assert prob.info().step_variant == variant
    assert wx <= TOL_STEP and wy <= TOL_STEP


@pytest.mark.parametrize("L,P,R", [(10, 16, 32), (8, 32, 8), (6, 8, 64), (7, 4, 64)])
def test_persistent_csr_solver_matches_per_step(sb, L, P, R):
    """The persistent CSR solver (one cooperative launch, grid barrier per
    step) and the per-step kernels give bit-identical runs, including the
    best-so-far readouts between stretches of steps (N = 343: ragged)."""
    pb, spec = lattice(L, L)
    out = []
    for sel in (1, 2, 11):  # per step; persistent caching items; persistent caching rows
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, L), **_params(kernel_select=sel, eval_every=37))
        sb.run(prob, 200, P, R, seed=L)
        assert prob.info().step_kernel == (0 if sel == 1 else 4)
        out.append((sb.get_state(prob)[:2], sb.get_energies(prob), sb.get_best(prob)))
    (xa, ya), ea, ba = out[0]
    for (xb, yb), eb, bb in out[1:]:
        assert np.array_equal(xa, xb) and np.array_equal(ya, yb)
        assert np.array_equal(ea[1], eb[1])
        for k in ba:
            assert np.array_equal(ba[k], bb[k]), k
    _check_best_with_readouts(sb, pb, prob, R, 200, 37)


def _check_best_with_readouts(sb, pb, prob, R, S, K):
    """With readouts every K steps the best-so-far comes from any readout:
    its energy is at most the final state's, its spins have that energy
    (oracle), and its step is one of the readout steps.  Equal energies keep
    the earlier configuration (strict improvement), so it need not be the
    final argmin when ground states are degenerate."""
    e, ei = sb.get_energies(prob)
    x, _, _ = sb.get_state(prob)
    spins = np.where(x >= 0, 1, -1).astype(np.int8)
    assert np.array_equal(ei, oracle.energies(pb, spins))
    best = sb.get_best(prob)
    steps = set(range(K - 1, S, K)) | {S - 1}
    for r in range(R):
        assert best["energy"][r] <= e[r].min()
        assert int(best["step"][r]) in steps
        assert oracle.energy_int(pb, best["spins"][r]) == best["energy_int"][r] == best["energy"][r]


@pytest.mark.parametrize("N,d,P,R,prec", [(600, 6, 16, 8, "bf16"), (500, 5, 8, 32, "fp32"), (300, 8, 32, 4, "fp32")])
def test_persistent_csr_solver_real_couplings(sb, N, d, P, R, prec):
    """Random regular graphs with real J (FP32 or BF16 product) and a field:
    the persistent solver (values cached beside the columns; W = 4 for
    R*P = 128, W = 8 for 256) in both cache modes equals the per-step kernels
    bit for bit."""
    pb, spec = regular(N, d, 7)
    out = []
    for sel in (1, 2, 11):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 4), **_params(precision=prec, kernel_select=sel,
                                                                          eval_every=25, gamma0=4.0 * P))
        sb.run(prob, 120, P, R, seed=3)
        assert prob.info().step_kernel == (0 if sel == 1 else 4)
        out.append((sb.get_state(prob)[:2], sb.get_energies(prob), sb.get_best(prob)))
    (xa, ya), ea, ba = out[0]
    for (xb, yb), eb, bb in out[1:]:
        assert np.array_equal(xa, xb) and np.array_equal(ya, yb)
        assert np.array_equal(ea[0], eb[0])
        for k in ba:
            assert np.array_equal(ba[k], bb[k]), k


def test_persistent_csr_solver_resume(sb):
    pb, spec = lattice(8, 2)
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(16, 2), **_params(kernel_select=2))
    sb.run(prob, 150, 16, 16, seed=4)
    xa = sb.get_state(prob)[0]
    sb.run_begin(prob, 150, 16, 16, seed=4)
    sb.run_advance(prob, 61)
    sb.run_advance(prob, 500)
    sb.run_finish(prob)
    assert np.array_equal(xa, sb.get_state(prob)[0])


def test_full_run_sk64_energies_exact(sb):
    pb, spec = sk(64, 0)
    prob = create(sb, spec)
    beta, alpha = workloads.linear_params(16)
    sb.set_schedule(prob, beta, alpha, **_params())
    sb.run(prob, 1000, 8, 16, seed=0)
    best = _check_energies_and_best(sb, pb, prob, 16, 8)
    assert np.all(best["step"] == 999)


def test_per_run_schedule_only_affects_its_run(sb):
    """The (alpha, beta) study batches a whole grid in one solve: run r's
    result depends only on its own (beta_r, alpha_r) and seed, bit for bit,
    whatever the other runs' parameters are."""
    pb, spec = lattice(6, 5)
    P, R, S = 16, 12, 200
    b1, a1 = workloads.autotune_params(R, 1)
    b2, a2 = workloads.autotune_params(R, 2)
    keep = np.arange(R) % 3 == 0
    b2[keep], a2[keep] = b1[keep], a1[keep]
    out = []
    for beta, alpha in ((b1, a1), (b2, a2)):
        prob = create(sb, spec)
        sb.set_schedule(prob, beta, alpha, **_params(gamma0=8.0))
        sb.run(prob, S, P, R, seed=5)
        out.append((sb.get_state(prob)[0], sb.get_best(prob)))
    assert np.array_equal(out[0][0][keep], out[1][0][keep])
    assert np.array_equal(out[0][1]["energy"][keep], out[1][1]["energy"][keep])
    assert not np.array_equal(out[0][0][~keep], out[1][0][~keep])


def test_schedule_tables_follow_schedule_and_shape_changes(sb):
    """The schedule tables are kept between runs of a handle and rebuilt when
    the schedule, the step count or the run shape changes: a handle run with
    schedule A, then B, then A again, then with another S and R equals fresh
    handles bit for bit."""
    pb, spec = lattice(6, 4)
    P = 16
    ba, aa = workloads.autotune_params(8, 1)
    bb, ab = workloads.autotune_params(8, 2)
    sched = {"A": (ba, aa, dict(gamma0=8.0)), "B": (bb, ab, dict(gamma0=32.0, jperp_enable=1)),
             "C": (ba[:4], aa[:4], dict(gamma0=8.0))}

    def solve(prob, key, S, R, set_schedule=True):
        b, a, kw = sched[key]
        if set_schedule:
            sb.set_schedule(prob, b, a, **_params(**kw))
        sb.run(prob, S, P, R, seed=3)
        return sb.get_state(prob)[0]

    reuse = create(sb, spec)
    seq = [("A", 120, 8), ("A", 120, 8), ("B", 120, 8), ("A", 120, 8), ("A", 90, 8), ("C", 90, 4)]
    last = None
    for key, S, R in seq:
        got = solve(reuse, key, S, R, set_schedule=key != last)  # the same schedule again: tables reused
        last = key
        assert np.array_equal(got, solve(create(sb, spec), key, S, R)), (key, S, R)


# ---------------------------------------------------------------- ballistic form f(x) = x
@pytest.mark.parametrize("case", ["lattice_pm1", "regular_f32_field", "dense_real", "dense_int", "ragged"])
def test_ballistic_per_step(sb, case):
    """f(x) = x (the bSB form of Sec. II A): one step from the same FP32 state
    against the oracle's bSB step, TOL_STEP per (run, replica)."""
    if case == "lattice_pm1":
        pb, spec = lattice(6, 2); P, R, prec = 32, 4, "auto"
    elif case == "regular_f32_field":
        pb, spec = regular(500, 6, 1); P, R, prec = 16, 8, "fp32"
    elif case == "dense_real":
        pb, spec = dense_real(100, 3); P, R, prec = 8, 4, "fp32"
    elif case == "dense_int":
        pb, spec = dense_int(300, 4); P, R, prec = 16, 9, "auto"
    else:
        pb, spec = lattice(3, 5); P, R, prec = 2, 3, "auto"
    wx, wy, amb, prob = _per_step(sb, pb, spec, P, R, 400, 30, prec=prec, variant=1, gamma0=4.0 * P)
    print("bSB %s per-step worst x %.2e y %.2e wall-ambiguous %d" % (case, wx, wy, amb))
    assert prob.info().step_kernel in ((7,) if spec[0] == "dense" else (6, 14))
    assert wx <= TOL_STEP and wy <= TOL_STEP


def test_ballistic_bf16_against_rounded_j(sb):
    pb, spec = regular(500, 6, 2)
    wx, wy, _, _ = _per_step(sb, pb, spec, 16, 8, 300, 30, prec="bf16", pb_oracle=pb.bf16(), variant=1,
                             gamma0=64.0)
    assert wx <= TOL_STEP and wy <= TOL_STEP


def test_ballistic_free_running_sk64(sb):
    """f is continuous in the ballistic form, so FP32 and FP64 trajectories
    separate only through the dynamics' own amplification: 100 steps at the
    stable schedule stay within TOL_TRAJ."""
    pb, spec = sk(64, 0)
    e = _free_running(sb, pb, spec, 8, 16, 1000, 100, gamma0=32.0, variant=1)
    print("bSB free-running max x %.2e y %.2e" % tuple(e.max(axis=0)))
    assert e.max() <= TOL_TRAJ


@pytest.mark.parametrize("dense", [False, True])
def test_ballistic_full_run_energies_and_resume(sb, dense):
    """A whole ballistic run: exact integer energies of the final spins, a
    valid best-so-far with readouts every 50 steps, and the same state when
    the run is split across begin/advance/finish."""
    pb, spec = sk(200, 5) if dense else lattice(8, 3)
    P, R, S = 8, 16, 300
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, 1), **_params(variant="ballistic", eval_every=50))
    sb.run(prob, S, P, R, seed=9)
    xa, ya, _ = sb.get_state(prob)
    _check_best_with_readouts(sb, pb, prob, R, S, 50)
    sb.run_begin(prob, S, P, R, seed=9)
    sb.run_advance(prob, 77)
    sb.run_advance(prob, S)
    sb.run_finish(prob)
    xb, yb, _ = sb.get_state(prob)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


def test_ballistic_set_state_resume(sb):
    """set_state restarts the f buffer from x: a run resumed from a dumped
    state equals the unbroken run bit for bit."""
    pb, spec = lattice(6, 4)
    P, R, S = 16, 8, 120
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, 2), **_params(variant="ballistic"))
    sb.run_begin(prob, S, P, R, seed=2)
    sb.run_advance(prob, 50)
    x50, y50, _ = sb.get_state(prob)
    sb.run_advance(prob, S)
    xa, ya, _ = sb.get_state(prob)
    sb.run_begin(prob, S, P, R, seed=777)
    sb.set_state(prob, x50, y50, 50)
    sb.run_advance(prob, S)
    xb, yb, _ = sb.get_state(prob)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


@pytest.mark.parametrize("case", ["lattice_pm1", "regular_f32_field", "regular_bf16", "general_p", "ragged",
                                  "runs_of_64", "runs_of_128"])
def test_ballistic_persistent_equals_per_step(sb, case):
    """The persistent CSR solver of the ballistic form (14) runs the same
    fused multiply-adds in the same order as the per-step kernel (6): whole
    runs, with readouts every 40 steps and split across begin/advance/finish,
    give the same state bit for bit, and the final energies are the oracle's
    integers of the returned spins."""
    P, R, prec = 16, 8, "auto"
    if case == "lattice_pm1":
        pb, spec = lattice(8, 3); P = 32
    elif case == "regular_f32_field":
        pb, spec = regular(700, 7, 3); prec = "fp32"
    elif case == "regular_bf16":
        pb, spec = regular(600, 5, 4); prec = "bf16"
    elif case == "general_p":
        pb, spec = lattice(6, 5); P, R = 6, 24
    elif case == "runs_of_64":
        pb, spec = lattice(6, 7); P, R = 64, 4
    elif case == "runs_of_128":
        pb, spec = regular(400, 6, 8); P, R, prec = 128, 2, "fp32"
    else:
        pb, spec = lattice(3, 6); P, R = 2, 3
    S = 200
    out = {}
    for sel in (1, 2):
        prob = create(sb, spec)
        sb.set_schedule(prob, *workloads.autotune_params(R, 4), **_params(variant="ballistic", precision=prec,
                                                                          eval_every=40, kernel_select=sel,
                                                                          gamma0=4.0 * P))
        sb.run(prob, S, P, R, seed=6)
        assert prob.info().step_kernel == (6 if sel == 1 else 14)
        x, y, _ = sb.get_state(prob)
        e, ei = sb.get_energies(prob)
        best = sb.get_best(prob)
        sb.run_begin(prob, S, P, R, seed=6)
        sb.run_advance(prob, 33)
        sb.run_advance(prob, S)
        sb.run_finish(prob)
        xb, yb, _ = sb.get_state(prob)
        assert np.array_equal(x, xb) and np.array_equal(y, yb)
        out[sel] = (x, y, ei, e, best["energy"])
    for a, b in zip(out[1], out[2]):
        assert np.array_equal(a, b)
    if pb.is_integer:
        spins = np.where(out[2][0] >= 0, 1, -1).astype(np.int8)
        assert np.array_equal(out[2][2], oracle.energies(pb, spins))


def test_ballistic_persistent_not_taken_when_items_overflow_the_cache(sb, monkeypatch):
    """With each warp's cache held to one item (test hook
    SBQA_TEST_PERSIST_CACHE=1) the ballistic solver's items no longer fit and
    kernel_select 2 keeps the per-step kernel."""
    pb, spec = lattice(8, 3)
    monkeypatch.setenv("SBQA_TEST_PERSIST_CACHE", "1")
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(64, 4), **_params(variant="ballistic", kernel_select=2,
                                                                       gamma0=128.0))
    sb.run(prob, 20, 32, 64, seed=6)
    assert prob.info().step_kernel == 6


def test_steps_zero_reads_initial_state(sb):
    pb, spec = lattice(4, 0)
    prob = create(sb, spec)
    sb.set_schedule(prob, **_params())
    sb.run(prob, 0, 8, 3, seed=5)
    best = _check_energies_and_best(sb, pb, prob, 3, 8)
    assert np.all(best["step"] == -1)
    x, _, _ = sb.get_state(prob)
    xo, _ = oracle.init_state(5, pb.n, 8, 3, 0.1)
    assert np.array_equal(x.astype(np.float64), xo)


def test_real_energies_sparse_and_dense(sb):
    for pb, spec, prec in (regular(300, 6, 3) + ("bf16",), dense_real(70, 2) + ("fp32",)):
        prob = create(sb, spec)
        sb.set_schedule(prob, **_params(precision=prec))
        sb.run(prob, 200, 4, 6, seed=1)
        _check_energies_and_best(sb, pb, prob, 6, 4)


def test_isolated_spins_and_single_spin(sb):
    # N = 1 (no couplings) and a lattice with extra isolated spins (empty rows)
    prob = sb.create_problem_csr(1, [0, 0], [], [], h=[0.5])
    sb.set_schedule(prob, **_params())
    sb.run(prob, 50, 2, 3, seed=2)
    best = sb.get_best(prob)
    assert np.all(best["energy"] == -0.5) and np.all(best["spins"] == 1)
    n, rp, col, val, _ = workloads.cubic_lattice(3, 0)
    rp2 = np.concatenate([rp, np.full(5, rp[-1])])
    pb = oracle.Problem.csr(n + 5, rp2, col, val, None)
    prob = sb.create_problem_csr(n + 5, rp2, col, val)
    sb.set_schedule(prob, **_params())
    sb.run(prob, 80, 4, 2, seed=3)
    _check_energies_and_best(sb, pb, prob, 2, 4)


def test_eval_every_best_so_far(sb):
    pb, spec = lattice(5, 3)
    prob = create(sb, spec)
    beta, alpha = workloads.autotune_params(8, 2)
    sb.set_schedule(prob, beta, alpha, **_params())
    sb.run(prob, 400, 8, 8, seed=9)
    final = sb.get_best(prob)
    sb.set_schedule(prob, beta, alpha, **_params(eval_every=50))
    sb.run(prob, 400, 8, 8, seed=9)
    kept = sb.get_best(prob)
    assert np.all(kept["energy"] <= final["energy"])
    assert set(kept["step"].tolist()) <= {49, 99, 149, 199, 249, 299, 349, 399}
    for r in range(8):
        assert oracle.energy_int(pb, kept["spins"][r]) == kept["energy"][r]


def test_best_energy_distribution_matches_oracle(sb):
    """256 runs x 8 replicas of the config-1 instance: final best energies of
    the GPU path and of the oracle are statistically indistinguishable."""
    scipy_stats = pytest.importorskip("scipy.stats")
    pb, spec = sk(64, 0)
    R, P, S = 256, 8, 1000
    beta, alpha = workloads.autotune_params(R, 11)
    prob = create(sb, spec)
    sb.set_schedule(prob, beta, alpha, **_params())
    sb.run(prob, S, P, R, seed=77)
    g = sb.get_best(prob)["energy"]
    o = oracle.run(pb, S, P, R, 77, beta, alpha)["best_energy"]
    rng = np.random.default_rng(0)
    both = np.concatenate([g, o])
    obs = abs(g.mean() - o.mean())
    perm = [abs(np.subtract(*rng.permutation(both).reshape(2, -1).mean(axis=1))) for _ in range(5000)]
    p_perm = (np.sum(np.array(perm) >= obs) + 1) / (len(perm) + 1)
    vals = np.unique(both)
    table = np.array([[np.sum(g == v) for v in vals], [np.sum(o == v) for v in vals]], dtype=float)
    # merge sparse bins (expected count < 5) from the low-energy end
    merged = []
    acc = np.zeros(2)
    for col in table.T:
        acc = acc + col
        if acc.sum() >= 10:
            merged.append(acc); acc = np.zeros(2)
    if acc.sum() > 0 and merged:
        merged[-1] = merged[-1] + acc
    table = np.array(merged).T
    p_chi = scipy_stats.chi2_contingency(table)[1] if table.shape[1] > 1 else 1.0
    print("mean gpu %.3f oracle %.3f p_perm %.3f p_chi2 %.3f" % (g.mean(), o.mean(), p_perm, p_chi))
    assert p_perm > 0.01 and p_chi > 0.01


# ---------------------------------------------------------------- determinism, resume, symmetry
def test_resume_is_bit_identical(sb):
    pb, spec = lattice(6, 4)
    beta, alpha = workloads.autotune_params(4, 4)
    prob = create(sb, spec)
    sb.set_schedule(prob, beta, alpha, **_params(eval_every=25))
    sb.run(prob, 300, 16, 4, seed=21)
    xa, ya, _ = sb.get_state(prob)
    ba = sb.get_best(prob)
    sb.run_begin(prob, 300, 16, 4, seed=21)
    sb.run_advance(prob, 113)
    xm, ym, sd = sb.get_state(prob)
    sb.set_state(prob, xm, ym, sd)  # host round trip of the checkpoint
    sb.run_advance(prob, 1000)
    sb.run_finish(prob)
    xb, yb, _ = sb.get_state(prob)
    bb = sb.get_best(prob)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)
    for k in ba:
        assert np.array_equal(ba[k], bb[k]), k


def test_negation_symmetry_bit_exact(sb):
    pb, spec = sk(40, 2)
    prob = create(sb, spec)
    sb.set_schedule(prob, **_params())
    sb.run_begin(prob, 500, 8, 4, seed=8)
    x0, y0, _ = sb.get_state(prob)
    sb.run_advance(prob, 150)
    xa, ya, _ = sb.get_state(prob)
    sb.run_begin(prob, 500, 8, 4, seed=8)
    sb.set_state(prob, -x0, -y0, 0)
    sb.run_advance(prob, 150)
    xb, yb, _ = sb.get_state(prob)
    assert np.array_equal(xa, -xb) and np.array_equal(ya, -yb)


def test_repeat_runs_deterministic(sb):
    pb, spec = regular(2000, 6, 5)
    prob = create(sb, spec)
    sb.set_schedule(prob, **_params(precision="bf16"))
    out = []
    for _ in range(2):
        sb.run(prob, 300, 16, 8, seed=4)
        out.append((sb.get_state(prob)[0], sb.get_energies(prob)[0]))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


# ---------------------------------------------------------------- full-size configurations, sampled
def _sampled_runs(sb, pb, spec, P, R, S, steps, runs, prec="auto", pb_oracle=None, kernels=None, gamma0=1.0):
    """Free-running parity of the listed runs against the oracle after `steps` steps, at the full size;
    `kernels` lists the step_kernel codes the autotuner must have picked (the kernel bench.py times)."""
    prob = create(sb, spec)
    beta, alpha = workloads.autotune_params(R, 1)
    p = _params(precision=prec, gamma0=gamma0)
    sb.set_schedule(prob, beta, alpha, **p)
    sb.run_begin(prob, S, P, R, seed=0)
    sb.run_advance(prob, steps)
    if kernels is not None:
        assert prob.info().step_kernel in kernels, prob.info().step_kernel
    xg, yg, _ = sb.get_state(prob)
    xi, yi = oracle.init_state(0, pb.n, P, max(runs) + 1, 0.1)
    worst = 0.0
    for r in runs:
        ref = oracle.run(pb_oracle or pb, S, P, 1, 0, beta[r:r + 1], alpha[r:r + 1], gamma0=gamma0, n_end=steps,
                         x0=xi[r:r + 1], y0=yi[r:r + 1], **_oracle_kwargs(p, pb))
        worst = max(worst, rel_err(xg[r:r + 1], ref["x"]), rel_err(yg[r:r + 1], ref["y"]))
    return worst


def test_full_size_lattice_L16_P32_R64(sb):
    """3D lattice L=16 (N=4096), P=32, R=64, 10^4-step schedule: runs 0, 37, 63 after 10 steps."""
    pb, spec = lattice(16, 0)
    assert _sampled_runs(sb, pb, spec, 32, 64, 10000, 10, [0, 37, 63]) <= TOL_TRAJ


def _sampled_per_step(sb, pb, spec, P, R, S, steps, runs, kernels, prec="auto", pb_oracle=None, gamma0=1.0):
    """The kernel the benchmark times, tied to the oracle at the full size: `steps` single-step launches,
    each compared on the sampled runs with one oracle step from the same FP32 state (TOL_STEP), then a
    fresh run of `steps` steps in one launch must equal the stepped state bit for bit.  `kernels` lists
    the step_kernel codes the autotuner must pick (the solver of the benchmark line)."""
    prob = create(sb, spec)
    beta, alpha = workloads.autotune_params(R, 1)
    p = _params(precision=prec, gamma0=gamma0)
    sb.set_schedule(prob, beta, alpha, **p)
    sb.run_begin(prob, S, P, R, seed=0)
    a, d, jp = oracle.schedule(S, P, R, beta, alpha, gamma0, p["delta_slope"], p["jperp_enable"])
    kw = _oracle_kwargs(p, pb)
    ref = pb_oracle or pb
    x, y, _ = sb.get_state(prob)
    worst = 0.0
    flips = []
    for n in range(steps):
        sb.run_advance(prob, 1)
        assert prob.info().step_kernel in kernels, prob.info().step_kernel
        xg, yg, _ = sb.get_state(prob)
        for r in runs:
            nf = _threshold_flips(x[r], x[r].astype(np.float64), d[n])
            if nf:
                flips.append((r, n, nf))
            xo, yo = oracle.step(ref, x[r].astype(np.float64), y[r].astype(np.float64), P, a[n], d[n], jp[r, n], **kw)
            amb = wall_ambiguous(xg[r:r + 1], xo[None])
            worst = max(worst, rel_err(xg[r:r + 1], xo[None]),
                        rel_err(np.where(amb, 0.0, yg[r:r + 1]), np.where(amb, 0.0, yo[None])))
        x, y = xg, yg
    if flips:
        print("FP32/FP64 threshold flips (run, step, count): %s" % flips[:20])
    sb.run_begin(prob, S, P, R, seed=0)
    sb.run_advance(prob, steps)  # one launch of the persistent solver for the whole stretch
    assert prob.info().step_kernel in kernels
    xb, yb, _ = sb.get_state(prob)
    assert np.array_equal(xb, x) and np.array_equal(yb, y)
    return worst


def test_full_size_lattice_L16_persistent_solver_against_oracle(sb):
    """Lattice L=16, P=32, R=64: the persistent CSR solver (step_kernel 4, the benchmark's kernel) against
    the oracle step by step on runs 0, 21 and 63 for 24 steps."""
    pb, spec = lattice(16, 0)
    assert _sampled_per_step(sb, pb, spec, 32, 64, 10000, 24, [0, 21, 63], kernels=(4,)) <= TOL_STEP


def test_full_size_lattice_energies(sb):
    pb, spec = lattice(16, 0)
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(64, 1), **_params())
    sb.run(prob, 40, 32, 64, seed=0)
    _check_energies_and_best(sb, pb, prob, 64, 32)


def test_full_size_dense_sk2000_exact(sb):
    """SK N=2000 +-1, P=32, R=32 (J.X = 2000x2000 @ 2000x1024), exact product: runs 0 and 31 after 5 steps."""
    pb, spec = sk(2000, 0)
    assert _sampled_runs(sb, pb, spec, 32, 32, 1000, 5, [0, 31], prec="exact") <= TOL_TRAJ


def test_full_size_dense_sk2000_persistent_solver_against_oracle(sb):
    """SK N=2000, P=32, R=32, exact product on a persistent tcgen05 solver (step_kernel 5, 8, 9, 15
    or 16, the benchmark's kernels; 15 and 16 with e2m1 operands) against the oracle step by step on
    runs 0 and 31 for 20 steps."""
    pb, spec = sk(2000, 0)
    assert _sampled_per_step(sb, pb, spec, 32, 32, 1000, 20, [0, 31], kernels=(5, 8, 9, 15, 16),
                             prec="exact") <= TOL_STEP


def test_full_size_dense_sk2000_energies(sb):
    """SK N=2000, P=32, R=32, exact product, 30 steps: the tensor-core readout energies of runs 0, 17
    and 31 (all replicas) equal the oracle's exact energies of the returned spins, and each run's best
    is the lowest of its replicas."""
    pb, spec = sk(2000, 0)
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(32, 1), **_params(precision="exact"))
    sb.run(prob, 30, 32, 32, seed=0)
    assert prob.info().step_kernel in (2, 5, 8, 9, 15, 16)
    e, ei = sb.get_energies(prob)
    x, _, _ = sb.get_state(prob)
    best = sb.get_best(prob)
    for r in (0, 17, 31):
        spins = np.where(x[r] >= 0, 1, -1)
        assert np.array_equal(ei[r], oracle.energies(pb, spins[None])[0])
        k = int(np.argmin(ei[r]))
        assert best["replica"][r] == k and best["energy"][r] == ei[r, k]
        assert np.array_equal(best["spins"][r], spins[k])


def test_full_size_regular_1e5_bf16(sb):
    """Random 6-regular N=1e5, J~N(0,1), h~N(0,0.1^2), BF16 product, P=16, R=8: runs 0 and 7 after 5 steps."""
    pb, spec = regular(100000, 6, 0)
    assert _sampled_runs(sb, pb, spec, 16, 8, 5000, 5, [0, 7], prec="bf16", pb_oracle=pb.bf16()) <= TOL_TRAJ


def test_full_size_regular_1e5_persistent_solver_against_oracle(sb):
    """Random 6-regular N=1e5, BF16 product, P=16, R=8 -- the benchmark's headline workload -- on the
    persistent CSR solver (step_kernel 4) against the oracle on the BF16-rounded J, step by step on runs
    0, 3 and 7 for 20 steps."""
    pb, spec = regular(100000, 6, 0)
    assert _sampled_per_step(sb, pb, spec, 16, 8, 5000, 20, [0, 3, 7], kernels=(4,), prec="bf16",
                             pb_oracle=pb.bf16()) <= TOL_STEP


# ---------------------------------------------------------------- errors that need a handle
def test_run_argument_errors(sb):
    pb, spec = sk(16, 0)
    prob = create(sb, spec)
    with pytest.raises(sb.SBQAError) as e:
        sb.run(prob, 10, 8, 2)
    assert e.value.status == sb.ERR_STATE
    sb.set_schedule(prob, *workloads.linear_params(3), **_params())
    for P, R, code in ((129, 3, sb.ERR_UNSUPPORTED), (0, 3, sb.ERR_INVALID_ARG), (8, 4, sb.ERR_INVALID_ARG),
                       (8, 0, sb.ERR_INVALID_ARG)):
        with pytest.raises(sb.SBQAError) as e:
            sb.run(prob, 10, P, R)
        assert e.value.status == code
    with pytest.raises(sb.SBQAError) as e:
        sb.get_best(prob)
    assert e.value.status == sb.ERR_STATE
    pr, sr = dense_real(20, 0)
    probr = create(sb, sr)
    with pytest.raises(sb.SBQAError) as e:
        sb.set_schedule(probr, **_params(precision="exact"))
    assert e.value.status == sb.ERR_UNSUPPORTED
    sb.set_schedule(prob, *workloads.linear_params(3), **_params(kernel_select=15))  # the largest selection
    for bad in (-1, 16):
        with pytest.raises(sb.SBQAError) as e:
            sb.set_schedule(prob, *workloads.linear_params(3), **_params(kernel_select=bad))
        assert e.value.status == sb.ERR_INVALID_ARG
