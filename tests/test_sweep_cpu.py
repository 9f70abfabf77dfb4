"""Host logic of the (alpha, beta) sensitivity study: the per-run schedule
layout of one batched solve and the optimality-gap table (Eq. 9)."""
import numpy as np

import bench


def test_sweep_layout_index_formula():
    alphas, betas, runs, reps = [0.5, 1.0, 2.0], [0.25, 1.5], 3, 4
    beta, alpha = bench.sweep_layout(alphas, betas, runs, reps)
    assert beta.size == alpha.size == len(alphas) * len(betas) * runs * reps
    for ia, a in enumerate(alphas):
        for ib, b in enumerate(betas):
            for q in range(runs):
                for t in range(reps):
                    r = ((ia * len(betas) + ib) * runs + q) * reps + t
                    assert alpha[r] == a and beta[r] == b


def test_sweep_table_best_of_repetitions_then_mean_gap():
    alphas, betas, runs, reps = [0.5, 1.0], [1.0, 2.0, 3.0], 2, 3
    E0 = -100.0
    rng = np.random.default_rng(0)
    e = rng.integers(-100, -60, size=len(alphas) * len(betas) * runs * reps).astype(float)
    g = bench.sweep_table(e, alphas, betas, runs, reps, E0)
    assert g.shape == (2, 3)
    for ia in range(2):
        for ib in range(3):
            best = []
            for q in range(runs):
                r0 = ((ia * 3 + ib) * runs + q) * reps
                best.append(min(e[r0:r0 + reps]))
            want = np.mean([(b - E0) / 100.0 for b in best])
            assert abs(g[ia, ib] - want) < 1e-15
    # a run that reaches E0 in any repetition contributes g = 0
    e2 = np.full_like(e, -80.0)
    e2[1] = E0
    g2 = bench.sweep_table(e2, alphas, betas, runs, reps, E0)
    assert g2[0, 0] == 0.5 * (0.0 + 0.2) and np.all(g2.ravel()[1:] == 0.2)
