"""The persistent CSR solver on instances whose items outnumber the
shared-memory cache: a warp caches the items that fit and reads the
neighbours of the rest from the ELL form every step (persistent mode 3).
The test hook SBQA_TEST_PERSIST_CACHE=k caps the cache at k items per warp,
so small instances take that path; the results equal the per-step kernels
bit for bit (which the parity tests tie to the oracle), and the best
energies equal the oracle's energies of the returned spins."""
import os

import numpy as np
import pytest

import oracle
import workloads
from sbqa_cases import create, lattice, regular

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as s
    return s


# (oracle problem, spec), P, R, precision: 128-column items on half warps with
# BF16 and FP32 values, 256-column items on whole warps (+-1), a ring of 6
# replicas in 8 columns
# replicas in 8 columns; every instance has more items than the grid's warps
# (4864 on 152 SMs) times the cap, so that items pass the cap on every warp
CASES = {
    "regular_bf16_half": (lambda: regular(20000, 6, 3), 16, 8, "bf16"),
    "regular_fp32_half": (lambda: regular(18000, 6, 4), 8, 16, "fp32"),
    "lattice_pm1_whole": (lambda: lattice(24, 5), 32, 8, "auto"),
    "lattice_ring6": (lambda: lattice(22, 6), 6, 32, "auto"),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("cap", [1, 2])
def test_items_beyond_cache_equal_per_step(sb, name, cap):
    make, P, R, prec = CASES[name]
    pb_o, spec = make()
    steps = 37
    out = {}
    for ks in (1, 2):  # per-step kernels, then the persistent solver with the capped cache
        pb = create(sb, spec)
        sb.set_schedule(pb, *workloads.autotune_params(R, 2), precision=prec, eval_every=9, kernel_select=ks)
        if ks == 2:
            os.environ["SBQA_TEST_PERSIST_CACHE"] = str(cap)
        try:
            sb.run(pb, steps, P, R, seed=21)
        finally:
            os.environ.pop("SBQA_TEST_PERSIST_CACHE", None)
        assert pb.info().step_kernel == (4 if ks == 2 else 0)
        x, y, _ = sb.get_state(pb)
        out[ks] = (x, y, sb.get_best(pb))
    assert np.array_equal(out[1][0], out[2][0]) and np.array_equal(out[1][1], out[2][1])
    b1, b2 = out[1][2], out[2][2]
    assert np.array_equal(b1["spins"], b2["spins"]) and np.array_equal(b1["energy"], b2["energy"])
    ref = oracle.energies(pb_o, b2["spins"])
    if pb_o.is_integer:
        assert np.array_equal(b2["energy_int"], ref)
    else:
        assert np.allclose(b2["energy"], ref, rtol=1e-12, atol=1e-9)
