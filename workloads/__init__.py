"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds none of the method's arithmetic: it only draws Ising
instances and per-run schedule parameters from seeded numpy generators.
The instance families stand in for the paper's benchmark sets (Zephyr,
QAC, tile planting, Pegasus-embedded lattices, HUBO), which are not
available here:

  sk_pm1            fully connected Sherrington-Kirkpatrick, J_ij = +-1
                    (p = 1/2), symmetric, zero diagonal, h = 0
  cubic_lattice     L x L x L periodic cubic lattice, 6 neighbours, J = +-1
                    (3D spin glass, Sec. III B 1 / Figs. 10-11 geometry)
  random_regular    random d-regular graph (configuration model, no self
                    loops or multi-edges), J ~ N(0, 1), h ~ N(0, sigma_h^2)
  autotune_params   per-run (beta, alpha) drawn uniformly from
                    [0.5, 1.5] x [0.5, 1.0] (the auto-tuning of Sec. II B)

Every generator returns plain numpy arrays: dense J (N x N float64) or CSR
(row_ptr int64, col int32, val float64) plus h (float64 or None).
"""
from __future__ import annotations

import numpy as np


def sk_pm1(n: int, seed: int = 0):
    """Dense SK instance with +-1 couplings; returns (J, h=None)."""
    rng = np.random.default_rng(seed)
    upper = np.triu(rng.choice(np.array([-1.0, 1.0]), size=(n, n)), k=1)
    J = upper + upper.T
    return J, None


def dense_to_csr(J):
    J = np.asarray(J)
    n = J.shape[0]
    rows, cols = np.nonzero(J)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), J[rows, cols].astype(np.float64)


def _csr_from_edges(n, ei, ej, w):
    """Symmetric CSR with sorted columns from undirected edges (i, j, w)."""
    rows = np.concatenate([ei, ej]); cols = np.concatenate([ej, ei]); vals = np.concatenate([w, w])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr), cols.astype(np.int32), vals.astype(np.float64)


def cubic_lattice(L: int, seed: int = 0):
    """Periodic L^3 lattice, J = +-1 on the 3 L^3 bonds; returns (n, row_ptr, col, val, h=None)."""
    rng = np.random.default_rng(seed)
    n = L ** 3
    idx = np.arange(n)
    x, y, z = idx % L, (idx // L) % L, idx // (L * L)
    ei, ej = [], []
    for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
        nb = ((x + dx) % L) + ((y + dy) % L) * L + ((z + dz) % L) * L * L
        ei.append(idx); ej.append(nb)
    ei = np.concatenate(ei); ej = np.concatenate(ej)
    w = rng.choice(np.array([-1.0, 1.0]), size=ei.size)
    if L <= 2:  # L <= 2 folds bonds onto each other; merge duplicates
        J = np.zeros((n, n))
        for a, b, c in zip(ei, ej, w):
            if a != b:
                J[a, b] += c; J[b, a] += c
        rp, col, val = dense_to_csr(J)
        return n, rp, col, val, None
    rp, col, val = _csr_from_edges(n, ei, ej, w)
    return n, rp, col, val, None


def random_regular(n: int, d: int = 6, seed: int = 0, sigma_h: float = 0.1, max_tries: int = 1000):
    """Random d-regular graph by the configuration model with rejection of
    self loops and multi-edges (stubs re-paired until simple).
    J ~ N(0,1) per edge, h ~ N(0, sigma_h^2).  Returns (n, row_ptr, col, val, h)."""
    if (n * d) % 2:
        raise ValueError("n * d must be even")
    rng = np.random.default_rng(seed)
    stubs = np.repeat(np.arange(n), d)
    for _ in range(max_tries):
        rng.shuffle(stubs)
        a, b = stubs[0::2].copy(), stubs[1::2].copy()
        # repair pass: re-pair bad pairs (self loops / duplicates) by swapping with random pairs
        for _rep in range(200):
            lo, hi = np.minimum(a, b), np.maximum(a, b)
            key = lo.astype(np.int64) * n + hi
            _, first = np.unique(key, return_index=True)
            bad = np.ones(a.size, dtype=bool); bad[first] = False
            bad |= (a == b)
            nb = int(bad.sum())
            if nb == 0:
                break
            bi = np.flatnonzero(bad)
            oj = rng.integers(0, a.size, size=nb)
            b[bi], b[oj] = b[oj].copy(), b[bi].copy()
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        if np.all(a != b) and np.unique(lo.astype(np.int64) * n + hi).size == a.size:
            w = rng.standard_normal(a.size)
            rp, col, val = _csr_from_edges(n, a, b, w)
            h = sigma_h * rng.standard_normal(n)
            return n, rp, col, val, h
    raise RuntimeError("configuration model did not produce a simple graph")


def autotune_params(R: int, seed: int = 0):
    """Per-run (beta, alpha) ~ U[0.5, 1.5] x U[0.5, 1.0]  (Sec. II B)."""
    rng = np.random.default_rng(seed)
    beta = rng.uniform(0.5, 1.5, size=R)
    alpha = rng.uniform(0.5, 1.0, size=R)
    return beta, alpha


def linear_params(R: int):
    """beta = 1, alpha = 1 for every run (the linear schedule)."""
    return np.ones(R), np.ones(R)


def random_dense_real(n: int, seed: int = 0, sigma_h: float = 0.0):
    """Dense symmetric J ~ N(0,1) off-diagonal, h ~ N(0, sigma_h^2)."""
    rng = np.random.default_rng(seed)
    upper = np.triu(rng.standard_normal((n, n)), k=1)
    h = sigma_h * rng.standard_normal(n) if sigma_h > 0 else None
    return upper + upper.T, h
