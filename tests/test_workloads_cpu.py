"""The seeded synthetic inputs (CPU only): each family has the structure its
recipe states -- symmetry, zero diagonal, value sets and distributions,
degrees, lattice geometry, simple graphs -- and the same seed gives the same
instance."""
import numpy as np
import pytest

import workloads


def _dense_from_csr(n, rp, col, val):
    J = np.zeros((n, n))
    for i in range(n):
        J[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    return J


def _check_csr(n, rp, col, val):
    assert rp.dtype == np.int64 and col.dtype == np.int32 and val.dtype == np.float64
    assert rp[0] == 0 and rp[-1] == col.size == val.size and np.all(np.diff(rp) >= 0)
    for i in range(n):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0), "columns sorted, no duplicates"
        assert not np.any(c == i), "no diagonal entry"
    J = _dense_from_csr(n, rp, col, val)
    assert np.array_equal(J, J.T), "symmetric"
    return J


def test_sk_pm1():
    J, h = workloads.sk_pm1(301, 4)
    assert h is None and J.shape == (301, 301)
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    off = J[~np.eye(301, dtype=bool)]
    assert set(np.unique(off)) == {-1.0, 1.0}
    assert abs(off.mean()) < 0.02  # p = 1/2: 45150 independent signs, sd of the mean 0.005
    assert np.array_equal(J, workloads.sk_pm1(301, 4)[0]) and not np.array_equal(J, workloads.sk_pm1(301, 5)[0])


@pytest.mark.parametrize("L", [3, 4, 7])
def test_cubic_lattice_geometry(L):
    n, rp, col, val, h = workloads.cubic_lattice(L, 2)
    assert n == L ** 3 and h is None
    J = _check_csr(n, rp, col, val)
    assert np.all(np.diff(rp) == 6), "6 neighbours on the periodic lattice"
    assert set(np.unique(val)) <= {-1.0, 1.0} and val.size == 6 * n
    for i in range(n):  # the neighbours are exactly the 6 sites one step away along an axis (mod L)
        x, y, z = i % L, (i // L) % L, i // (L * L)
        want = set()
        for d in (-1, 1):
            want.add(((x + d) % L) + y * L + z * L * L)
            want.add(x + ((y + d) % L) * L + z * L * L)
            want.add(x + y * L + ((z + d) % L) * L * L)
        assert set(np.flatnonzero(J[i])) == want


def test_cubic_lattice_small_folds_bonds():
    """L = 2: the +1 and -1 steps reach the same site, so bonds merge (values
    in {-2, 0, 2}, zeros dropped) and the matrix stays symmetric."""
    n, rp, col, val, _ = workloads.cubic_lattice(2, 1)
    _check_csr(n, rp, col, val)
    assert set(np.unique(val)) <= {-2.0, 2.0} and np.all(np.diff(rp) <= 3)


@pytest.mark.parametrize("n,d", [(1000, 6), (501, 4), (64, 3)])
def test_random_regular_is_simple_and_regular(n, d):
    if (n * d) % 2:
        with pytest.raises(ValueError):
            workloads.random_regular(n, d, 0)
        return
    n2, rp, col, val, h = workloads.random_regular(n, d, 7, 0.1)
    assert n2 == n
    _check_csr(n, rp, col, val)  # simple: no self loops, no duplicate columns, symmetric values
    assert np.all(np.diff(rp) == d)
    w = val[np.repeat(np.arange(n), d) < col]  # one value per edge
    assert w.size == n * d // 2
    if w.size > 1000:
        assert abs(w.mean()) < 0.15 and abs(w.std() - 1.0) < 0.1  # J ~ N(0, 1)
    assert h.shape == (n,) and abs(h.std() - 0.1) < 0.03  # h ~ N(0, 0.1^2)


def test_autotune_and_linear_params():
    beta, alpha = workloads.autotune_params(4000, 3)
    assert beta.min() >= 0.5 and beta.max() < 1.5 and alpha.min() >= 0.5 and alpha.max() < 1.0
    assert abs(beta.mean() - 1.0) < 0.02 and abs(alpha.mean() - 0.75) < 0.01
    b1, a1 = workloads.linear_params(5)
    assert np.all(b1 == 1.0) and np.all(a1 == 1.0)


def test_dense_to_csr_round_trip():
    J, _ = workloads.random_dense_real(40, 1)
    J[np.abs(J) < 0.5] = 0.0
    rp, col, val = workloads.dense_to_csr(J)
    assert np.array_equal(_check_csr(40, rp, col, val), J)
