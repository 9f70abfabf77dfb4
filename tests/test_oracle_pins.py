"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one oracle function to a published value, a closed form, a
symmetry of the equations, a special case that reduces to another
formulation, or brute force -- chosen so that a dropped term, a wrong sign,
a wrong replica index or a missing 1/P factor fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- RNG
def test_splitmix64_published_vector():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    for idx, val in rows:
        assert oracle.splitmix64(1234567, int(idx)) == int(val)


def test_uniform_f32_endpoints_and_grid():
    amp = 0.1
    assert oracle.uniform_f32(0, amp) == np.float32(-1.0) * np.float32(amp)
    top = ((1 << 24) - 1) << 40
    assert oracle.uniform_f32(top, amp) == np.float32((2 ** 23 - 1) / 2 ** 23) * np.float32(amp)
    assert oracle.uniform_f32(1 << 63, amp) == 0.0
    assert oracle.uniform_f32(0, 1.0) == -1.0


def test_init_state_range_stats_and_run_prefix():
    x, y = oracle.init_state(7, 33, 4, 6, 0.1)
    for a in (x, y):
        assert a.min() >= -0.1 - 1e-9 and a.max() < 0.1
        assert abs(a.mean()) < 0.01
        assert np.all(a == a.astype(np.float32).astype(np.float64))
    assert not np.array_equal(x, y)
    # runs are laid out first in the counter, so a smaller R is a prefix
    xs, ys = oracle.init_state(7, 33, 4, 2, 0.1)
    assert np.array_equal(xs, x[:2]) and np.array_equal(ys, y[:2])
    # a different seed gives a different state
    x2, _ = oracle.init_state(8, 33, 4, 6, 0.1)
    assert not np.array_equal(x, x2)


# ---------------------------------------------------------------- bf16
def test_round_bf16_ties_and_library():
    r = oracle.round_bf16
    assert r(1.0) == 1.0
    assert r(1.0 + 2 ** -8) == 1.0                      # tie -> even
    assert r(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6         # tie -> even (up)
    assert r(1.0 + 2 ** -8 + 2 ** -20) == 1.0 + 2 ** -7  # above the tie
    assert r(-1.0 - 2 ** -8) == -1.0
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(0).standard_normal(4000).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(r(v.astype(np.float64)), ref)


# ---------------------------------------------------------------- schedule
@pytest.mark.parametrize("beta,gam,P", [(1.0, 1.0, 8), (0.5, 3.0, 32), (1.5, 1e-5, 16), (0.7, 20.0, 4)])
def test_jperp_from_trotter_matrix_element(beta, gam, P):
    """J_perp = b / beta where exp(a + b) and exp(a - b) are the diagonal and
    off-diagonal elements of exp(theta sigma_x), theta = beta Gamma / P
    (Supplement Eqs. S6-S9, S12), evaluated with a matrix exponential."""
    theta = beta * gam / P
    M = scipy.linalg.expm(np.array([[0.0, theta], [theta, 0.0]]))
    b = 0.5 * math.log(M[0, 0] / M[0, 1])
    assert oracle.jperp(beta, gam, P) == pytest.approx(b / beta, rel=1e-9)
    # the coth form of Eq. S12 as a second expression
    assert oracle.jperp(beta, gam, P) == pytest.approx(
        math.log(1.0 / math.tanh(theta)) / (2 * beta), rel=1e-12)


def test_gamma_schedule_closed_forms():
    assert oracle.gamma(2.0, 1.0, 0.0) == pytest.approx(2.0 * (1 + 1e-5), rel=1e-15)
    assert oracle.gamma(2.0, 0.7, 1.0) == pytest.approx(2.0e-5, rel=1e-12)
    assert oracle.gamma(1.0, 0.5, 0.75) == pytest.approx(0.5 + 1e-5, rel=1e-12)
    assert oracle.gamma(3.0, 1.0, 0.25) == pytest.approx(3.0 * (0.75 + 1e-5), rel=1e-12)


def test_schedule_tables():
    S, P, R = 50, 8, 3
    beta = np.array([0.5, 1.0, 1.5]); alpha = np.array([0.5, 0.75, 1.0])
    a, d, jp = oracle.schedule(S, P, R, beta, alpha, gamma0=1.0)
    assert np.array_equal(a, np.arange(S) / S)
    assert np.allclose(d, 0.7 * np.arange(S + 1) / S, rtol=0, atol=1e-15)
    assert np.all(np.isfinite(jp)) and np.all(jp > 0)
    assert np.all(np.diff(jp, axis=1) > 0)  # Gamma_x falls, coupling grows
    # last step is tau = (S-1)/S; the 1e-5 keeps the endpoint finite
    for r in range(R):
        assert jp[r, 0] == pytest.approx(oracle.jperp(beta[r], 1.0 + 1e-5, P), rel=1e-12)
    _, _, jp0 = oracle.schedule(S, P, R, beta, alpha, jperp_enable=False)
    assert np.all(jp0 == 0)


# ---------------------------------------------------------------- f
def test_threshold_function_cases():
    assert oracle.f(0.3, 0.3) == 0.0            # |x| == Delta -> 0 (inclusive)
    assert oracle.f(-0.3, 0.3) == 0.0
    assert oracle.f(0.30001, 0.3) == 1.0
    assert oracle.f(-0.30001, 0.3) == -1.0
    assert oracle.f(0.0, 0.0) == 0.0            # Delta(0) = 0: f = sign with f(0) = 0
    assert oracle.f(1e-30, 0.0) == 1.0
    assert oracle.f(-1e-30, 0.0) == -1.0
    assert oracle.f(0.123, 0.7, variant=1) == 0.123
    # compared in FP64: a value above Delta by far less than an FP32 ulp is above it
    assert oracle.f(0.3 + 1e-12, 0.3) == 1.0
    assert oracle.f(-(0.3 + 1e-12), 0.3) == -1.0
    assert oracle.f(0.3 - 1e-12, 0.3) == 0.0


# ---------------------------------------------------------------- force = -dH/dq
def _hamiltonian(J, h, x, y, P, a, a0, c0, jp):
    """Eq. 4 with q -> x, p -> y, the replica count written P:
    H = sum_{i,k} [a0/(2P) p^2 + (a0-a)/(2P) q^2 - (c0/P)(h_i q_{ik} + 1/2 sum_j J_ij q_ik q_jk)
                   - J_perp q_{i,k} q_{i,k+1}], k periodic."""
    kin = a0 / (2 * P) * np.sum(y ** 2)
    pot = (a0 - a) / (2 * P) * np.sum(x ** 2)
    prob = -(c0 / P) * (np.sum(x @ h) + 0.5 * np.einsum("ki,ij,kj->", x, J, x))
    ring = -jp * np.sum(x * np.roll(x, -1, axis=0))
    return kin + pot + prob + ring


@pytest.mark.parametrize("P", [1, 2, 3, 8])
def test_force_is_minus_gradient_of_hamiltonian_bsb(P):
    """With f(x) = x the right-hand side of Eq. 7 must be -dH/dq of Eq. 4."""
    rng = np.random.default_rng(P)
    N = 7
    J, _ = workloads.random_dense_real(N, seed=3)
    h = rng.standard_normal(N)
    pb = oracle.Problem.dense(J, h)
    x = rng.uniform(-0.9, 0.9, (P, N)); y = np.zeros((P, N))
    a0, c0, a, jp = 1.0, 0.37, 0.31, 0.83
    F = oracle.force(pb, x, P, a, 0.0, jp, a0=a0, c0=c0, variant=1)
    eps = 1e-6
    G = np.zeros_like(x)
    for k in range(P):
        for i in range(N):
            xp = x.copy(); xp[k, i] += eps
            xm = x.copy(); xm[k, i] -= eps
            G[k, i] = (_hamiltonian(J, h, xp, y, P, a, a0, c0, jp)
                       - _hamiltonian(J, h, xm, y, P, a, a0, c0, jp)) / (2 * eps)
    assert np.allclose(F, -G, rtol=1e-7, atol=1e-8)


def test_force_dsb_equals_bsb_at_walls_and_drops_coupling_below_threshold():
    rng = np.random.default_rng(1)
    P, N = 4, 9
    J, _ = workloads.random_dense_real(N, seed=5)
    pb = oracle.Problem.dense(J, rng.standard_normal(N))
    xw = rng.choice([-1.0, 1.0], size=(P, N))
    args = dict(a0=1.0, c0=0.2)
    assert np.allclose(oracle.force(pb, xw, P, 0.4, 0.5, 0.6, variant=0, **args),
                       oracle.force(pb, xw, P, 0.4, 0.5, 0.6, variant=1, **args), rtol=0, atol=1e-14)
    xs = rng.uniform(-0.3, 0.3, (P, N))  # all |x| <= Delta -> J term vanishes
    pb0 = oracle.Problem.dense(np.zeros((N, N)), pb.h)
    assert np.allclose(oracle.force(pb, xs, P, 0.4, 0.35, 0.6, **args),
                       oracle.force(pb0, xs, P, 0.4, 0.35, 0.6, **args), rtol=0, atol=1e-15)


def test_step_free_motion_and_wall():
    """J = h = 0, a = a0, J_perp = 0: no force, so y is unchanged and
    x advances by dt (a0/P) y (dq/dt = dH/dp, Eq. 6).  A step that carries x
    past 1 clamps it to sign(x) and zeroes y (wall rule after Eq. 3)."""
    P, N = 4, 3
    pb = oracle.Problem.dense(np.zeros((N, N)))
    x = np.full((P, N), 0.25); y = np.full((P, N), 0.5); y[0, 0] = 100.0; y[1, 1] = -100.0
    xn, yn = oracle.step(pb, x, y, P, 1.0, 0.0, 0.0, a0=1.0, c0=0.3, dt=0.5)
    exp_x = 0.25 + 0.5 * (1.0 / P) * y
    exp_y = y.copy()
    exp_x[0, 0], exp_y[0, 0] = 1.0, 0.0
    exp_x[1, 1], exp_y[1, 1] = -1.0, 0.0
    assert np.array_equal(xn, exp_x) and np.array_equal(yn, exp_y)


def test_bsb_energy_conserved_for_small_dt():
    """Symplectic Euler on Eqs. 6-7 with f(x) = x and frozen parameters keeps
    the Eq. 4 energy within O(dt) of its start (no walls reached)."""
    rng = np.random.default_rng(2)
    P, N = 4, 6
    J, _ = workloads.random_dense_real(N, seed=8)
    h = 0.1 * rng.standard_normal(N)
    pb = oracle.Problem.dense(J, h)
    x = rng.uniform(-0.05, 0.05, (P, N)); y = rng.uniform(-0.05, 0.05, (P, N))
    a0, c0, a, jp, dt = 1.0, 0.1, 0.2, 0.05, 0.01
    H0 = _hamiltonian(J, h, x, y, P, a, a0, c0, jp)
    drift = 0.0
    for _ in range(2000):
        x, y = oracle.step(pb, x, y, P, a, 0.0, jp, a0=a0, c0=c0, dt=dt, variant=1)
        assert np.all(np.abs(x) < 1)
        drift = max(drift, abs(_hamiltonian(J, h, x, y, P, a, a0, c0, jp) - H0))
    assert drift < 0.02 * abs(H0)


# ---------------------------------------------------------------- reductions and symmetries
def _plain_sb(J, h, x, y, S, a0, c0, dt, delta_slope):
    """Plain SB (Eq. 3) with the thresholded f, symplectic Euler, wall; one replica."""
    x = x.copy(); y = y.copy()
    for n in range(S):
        tau = n / S
        d = delta_slope * tau
        fx = np.where(np.abs(x) <= d, 0.0, np.sign(x))
        y = y + dt * (-(a0 - tau) * x + c0 * (J @ fx + (h if h is not None else 0.0)))
        x = x + dt * a0 * y
        over = np.abs(x) > 1
        x[over] = np.sign(x[over]); y[over] = 0.0
    return x, y


def test_jperp_zero_reduces_to_plain_sb_with_step_dt_over_P():
    """With J_perp = 0 each replica of Eqs. 6-7 is plain SB (Eq. 3) with the
    time step dt / P."""
    N, P, R, S = 12, 4, 2, 60
    J, _ = workloads.sk_pm1(N, seed=4)
    h = np.random.default_rng(0).standard_normal(N) * 0.3
    pb = oracle.Problem.dense(J, h)
    beta, alpha = workloads.autotune_params(R, 0)
    res = oracle.run(pb, S, P, R, 11, beta, alpha, c0=0.3, dt=0.5, jperp_enable=False)
    x0, y0 = oracle.init_state(11, N, P, R, 0.1)
    for r in range(R):
        for k in range(P):
            xs, ys = _plain_sb(J, h, x0[r, k], y0[r, k], S, 1.0, 0.3, 0.5 / P, 0.7)
            assert np.allclose(res["x"][r, k], xs, rtol=0, atol=1e-12)
            assert np.allclose(res["y"][r, k], ys, rtol=0, atol=1e-12)


def _small_case(h=True):
    N, P, R, S = 10, 6, 2, 80
    J, _ = workloads.sk_pm1(N, seed=9)
    hv = np.random.default_rng(1).integers(-2, 3, N).astype(float) if h else None
    return oracle.Problem.dense(J, hv), N, P, R, S


def test_negation_symmetry_at_zero_field():
    pb, N, P, R, S = _small_case(h=False)
    beta, alpha = workloads.autotune_params(R, 1)
    x0, y0 = oracle.init_state(3, N, P, R, 0.1)
    a = oracle.run(pb, S, P, R, 0, beta, alpha, x0=x0, y0=y0, n_traj=S)
    b = oracle.run(pb, S, P, R, 0, beta, alpha, x0=-x0, y0=-y0, n_traj=S)
    assert np.array_equal(a["traj_x"], -b["traj_x"]) and np.array_equal(a["traj_y"], -b["traj_y"])
    assert np.array_equal(a["best_energy"], b["best_energy"])


def test_replica_ring_shift_and_reflection():
    """The replica axis is a periodic ring (Supplement Eq. S3): relabelling
    k -> k+1 or k -> -k maps trajectories onto each other exactly."""
    pb, N, P, R, S = _small_case()
    beta, alpha = workloads.autotune_params(R, 2)
    x0, y0 = oracle.init_state(5, N, P, R, 0.1)
    base = oracle.run(pb, S, P, R, 0, beta, alpha, x0=x0, y0=y0, n_traj=S)
    sh = oracle.run(pb, S, P, R, 0, beta, alpha, x0=np.roll(x0, 1, axis=1), y0=np.roll(y0, 1, axis=1), n_traj=S)
    assert np.array_equal(np.roll(base["traj_x"], 1, axis=2), sh["traj_x"])
    ref = oracle.run(pb, S, P, R, 0, beta, alpha, x0=x0[:, ::-1], y0=y0[:, ::-1], n_traj=S)
    assert np.array_equal(base["traj_x"][:, :, ::-1], ref["traj_x"])
    assert np.array_equal(base["traj_y"][:, :, ::-1], ref["traj_y"])


def test_spin_relabelling_integer_instance():
    pb, N, P, R, S = _small_case()
    perm = np.random.default_rng(3).permutation(N)
    J = pb.to_dense(); h = pb.h
    pbp = oracle.Problem.dense(J[np.ix_(perm, perm)], h[perm])
    beta, alpha = workloads.autotune_params(R, 3)
    x0, y0 = oracle.init_state(6, N, P, R, 0.1)
    a = oracle.run(pb, S, P, R, 0, beta, alpha, x0=x0, y0=y0)
    b = oracle.run(pbp, S, P, R, 0, beta, alpha, x0=x0[:, :, perm], y0=y0[:, :, perm])
    assert np.array_equal(a["x"][:, :, perm], b["x"])
    assert np.array_equal(a["energy"], b["energy"])


def test_runs_are_independent_prefix():
    pb, N, P, R, S = _small_case()
    beta, alpha = workloads.autotune_params(5, 4)
    big = oracle.run(pb, S, P, 5, 21, beta, alpha)
    small = oracle.run(pb, S, P, 2, 21, beta[:2], alpha[:2])
    assert np.array_equal(big["x"][:2], small["x"])
    assert np.array_equal(big["best_energy"][:2], small["best_energy"])


def test_resume_at_step_boundary_is_bit_identical():
    pb, N, P, R, S = _small_case()
    beta, alpha = workloads.autotune_params(R, 5)
    full = oracle.run(pb, S, P, R, 2, beta, alpha, eval_every=7)
    first = oracle.run(pb, S, P, R, 2, beta, alpha, n_end=33, eval_every=7)
    second = oracle.run(pb, S, P, R, 2, beta, alpha, n_begin=33, x0=first["x"], y0=first["y"],
                        eval_every=7, best=first)
    for key in ("x", "y", "energy", "best_energy", "best_k", "best_step", "best_spins"):
        assert np.array_equal(full[key], second[key]), key


# ---------------------------------------------------------------- energies
def test_energy_hand_example():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "energy_3spin.txt"))
             if l.strip() and not l.startswith("#")]
    J = np.zeros((3, 3)); h = s = E = None
    for t in lines:
        if t[0] == "J":
            i, j, v = int(t[1]), int(t[2]), float(t[3]); J[i, j] = J[j, i] = v
        elif t[0] == "h":
            h = np.array([float(v) for v in t[1:]])
        elif t[0] == "s":
            s = np.array([int(v) for v in t[1:]])
        elif t[0] == "E":
            E = float(t[1])
    assert oracle.energy(oracle.Problem.dense(J, h), s) == E


@pytest.mark.parametrize("N", [2, 5, 8, 11])
def test_brute_force_closed_forms(N):
    ferro = oracle.Problem.dense(np.ones((N, N)) - np.eye(N))
    assert oracle.brute_force(ferro)[0] == -N * (N - 1) / 2
    anti = oracle.Problem.dense(-(np.ones((N, N)) - np.eye(N)))
    # E = ((sum s)^2 - N) / 2, minimised by |sum s| = N mod 2
    assert oracle.brute_force(anti)[0] == ((N % 2) - N) / 2
    h = np.random.default_rng(N).standard_normal(N)
    field = oracle.Problem.dense(np.zeros((N, N)), h)
    assert oracle.brute_force(field)[0] == pytest.approx(-np.abs(h).sum(), rel=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_ring_closed_form(seed):
    """Ring of N spins with couplings J_l: E0 = -sum|J| + 2 min|J| when the
    product of the signs is negative (frustrated), else -sum|J|."""
    rng = np.random.default_rng(seed)
    N = 9
    w = rng.uniform(0.5, 2.0, N) * rng.choice([-1, 1], N)
    J = np.zeros((N, N))
    for l in range(N):
        J[l, (l + 1) % N] = J[(l + 1) % N, l] = w[l]
    e0 = -np.abs(w).sum() + (2 * np.abs(w).min() if np.prod(np.sign(w)) < 0 else 0.0)
    assert oracle.brute_force(oracle.Problem.dense(J))[0] == pytest.approx(e0, rel=1e-12)


def test_energy_int_matches_float_and_flip_symmetry():
    J, _ = workloads.sk_pm1(40, seed=2)
    pb = oracle.Problem.dense(J)
    rng = np.random.default_rng(0)
    for _ in range(20):
        s = rng.choice([-1, 1], 40).astype(np.int8)
        assert oracle.energy_int(pb, s) == oracle.energy(pb, s)
        assert oracle.energy_int(pb, s) == oracle.energy_int(pb, -s)


def test_readout_best_is_min_and_ties_take_lowest_replica():
    pb, N, P, R, S = _small_case()
    beta, alpha = workloads.autotune_params(R, 6)
    res = oracle.run(pb, S, P, R, 8, beta, alpha)
    for r in range(R):
        assert res["best_energy"][r] == res["energy"][r].min()
        assert res["best_k"][r] == int(np.argmin(res["energy"][r]))
        k = res["best_k"][r]
        s = np.where(res["x"][r, k] >= 0, 1, -1)
        assert np.array_equal(res["best_spins"][r], s)
    # identical replicas: the tie goes to k = 0
    x0, y0 = oracle.init_state(1, N, 1, R, 0.1)
    same = oracle.run(pb, S, P, R, 0, beta, alpha, x0=np.repeat(x0, P, 1), y0=np.repeat(y0, P, 1))
    assert np.all(same["best_k"] == 0)


def test_long_runs_reach_brute_force_ground_state():
    """R * P = 256 replicas of SBQA on small SK instances reach the exhaustive
    ground state (success-probability pin, not bit-exact)."""
    for seed in range(3):
        J, _ = workloads.sk_pm1(16, seed)
        pb = oracle.Problem.dense(J)
        e0, s0 = oracle.brute_force(pb)
        assert oracle.energy(pb, s0) == e0
        beta, alpha = workloads.autotune_params(32, seed)
        res = oracle.run(pb, 1000, 8, 32, seed, beta, alpha, gamma0=16.0)
        assert res["best_energy"].min() == e0
        assert np.all(res["best_energy"] >= e0)


# ---------------------------------------------------------------- metrics
def test_gap_and_tte_closed_forms():
    assert oracle.gap(-90.0, -100.0) == pytest.approx(0.1)
    assert oracle.tte(2.0, 0.5) == pytest.approx(2.0 * math.log(0.01) / math.log(0.5))
    assert oracle.tte(2.0, 0.0) == math.inf
    assert oracle.tte(2.0, 0.995) == 2.0
    assert oracle.tte(1.0, 0.9) == pytest.approx(2.0)  # log(0.01)/log(0.1) = 2


def test_c0_auto_closed_forms():
    N = 50
    J, _ = workloads.sk_pm1(N, 0)
    assert oracle.c0_auto(oracle.Problem.dense(J)) == pytest.approx(0.5 / math.sqrt(N - 1))
    n, rp, col, val, h = workloads.cubic_lattice(4, 0)
    assert oracle.c0_auto(oracle.Problem.csr(n, rp, col, val)) == pytest.approx(0.5 / math.sqrt(6))
