"""Shared builders for the GPU parity tests: the same seeded instance as an
oracle problem and as a library handle, plus comparison helpers."""
import numpy as np

import oracle
import workloads


def sk(n, seed=0):
    J, h = workloads.sk_pm1(n, seed)
    return oracle.Problem.dense(J, h), ("dense", J, h)


def lattice(L, seed=0):
    n, rp, col, val, h = workloads.cubic_lattice(L, seed)
    return oracle.Problem.csr(n, rp, col, val, h), ("csr", n, rp, col, val, h)


def regular(n, d=6, seed=0, sigma_h=0.1):
    n, rp, col, val, h = workloads.random_regular(n, d, seed, sigma_h)
    return oracle.Problem.csr(n, rp, col, val, h), ("csr", n, rp, col, val, h)


def dense_real(n, seed=0, sigma_h=0.2):
    J, h = workloads.random_dense_real(n, seed, sigma_h)
    return oracle.Problem.dense(J, h), ("dense", J, h)


def dense_int(n, seed=0, jmax=3):
    rng = np.random.default_rng(seed)
    up = np.triu(rng.integers(-jmax, jmax + 1, (n, n)).astype(float), 1)
    h = rng.integers(-2, 3, n).astype(float)
    J = up + up.T
    return oracle.Problem.dense(J, h), ("dense", J, h)


def create(sb, spec):
    if spec[0] == "dense":
        return sb.create_problem_dense(spec[1], spec[2])
    _, n, rp, col, val, h = spec
    return sb.create_problem_csr(n, rp, col, val, h)


def rel_err(a, b):
    """max over (r, k) of ||a - b||_inf / max(||b||_inf, 1e-3), arrays (R, P, N)."""
    num = np.abs(a - b).max(axis=-1)
    den = np.maximum(np.abs(b).max(axis=-1), 1e-3)
    return float((num / den).max())


def wall_ambiguous(xg, xo):
    """Elements where the strict wall test |x| > 1 can decide differently in
    FP32 and FP64: both positions lie within rounding of the wall and at
    least one sits exactly on it -- clamped, or an FP32 position that rounded
    to exactly 1 without being clamped while the FP64 one landed just above 1
    and was.  Those elements are excluded from the y comparison (their x
    agree to 4e-6)."""
    on_wall = (np.abs(xg) == 1.0) | (np.abs(xo) == 1.0)
    near_g = np.abs(np.abs(xg) - 1.0) < 4e-6
    near_o = np.abs(np.abs(xo) - 1.0) < 4e-6
    return on_wall & near_g & near_o
