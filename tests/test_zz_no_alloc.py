"""sbqa_energies_csr_noalloc against the solver's own readout and the oracle.

The entry point serves callers that cannot allocate device memory where they
need energies (inside a CUDA graph capture, in loops that must not block in
the allocator, under a host-owned memory pool): it takes the caller's device
buffers and keeps its partial sums in a fixed array inside the library.
This file is collected last so that a stop at the first failure has already
run every other test; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as sb
    return sb, torch


def _solver_energies(sb, create, P, R, seed, steps, prec="auto"):
    """Energies and final spins from the existing entry points."""
    prob = create()
    sb.set_schedule(prob, *workloads.autotune_params(R, seed), precision=prec)
    sb.run(prob, steps, P, R, seed=seed)
    e, ei = sb.get_energies(prob)
    x, _, _ = sb.get_state(prob)
    spins = np.where(x >= 0, 1, -1).astype(np.int8).reshape(R * P, -1)  # [config][spin]
    return e.reshape(-1), ei.reshape(-1), spins


def _dev(torch, a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def test_noalloc_integer_energies_match_solver_two_calls(env):
    sb, torch = env
    n, rp, col, val, _ = workloads.cubic_lattice(8, 1)
    h = np.random.default_rng(0).integers(-2, 3, n).astype(float)
    create = lambda: sb.create_problem_csr(n, rp, col, val, h)  # noqa: E731
    d_rp, d_col = _dev(torch, rp, np.int32), _dev(torch, col, np.int32)
    d_val, d_h = _dev(torch, val, np.int32), _dev(torch, h, np.int64)
    for seed, (P, R) in ((3, (8, 6)), (4, (16, 5))):  # two calls in a row, different sizes
        e_ref, ei_ref, spins = _solver_energies(sb, create, P, R, seed, 150)
        count = spins.shape[0]
        ld = count + 3  # a row stride wider than the configuration count
        sp = np.zeros((n, ld), dtype=np.int8)
        sp[:, :count] = spins.T
        d_sp = _dev(torch, sp, np.int8)
        out_i = torch.full((count,), 7, dtype=torch.int64, device="cuda")
        out_f = torch.full((count,), 7.0, dtype=torch.float64, device="cuda")
        sb.energies_csr_noalloc(n, d_rp.data_ptr(), d_col.data_ptr(), d_sp.data_ptr(), ld, count,
                                val_i32=d_val.data_ptr(), h_i64=d_h.data_ptr(),
                                energy_int=out_i.data_ptr(), energy=out_f.data_ptr())
        torch.cuda.synchronize()
        assert np.array_equal(out_i.cpu().numpy(), ei_ref)
        assert np.array_equal(out_f.cpu().numpy(), e_ref)
        # and the exact integer energies of the oracle (Eq. 4 sign) on the same spins
        assert np.array_equal(out_i.cpu().numpy(), oracle.energies(oracle.Problem.csr(n, rp, col, val, h), spins))


def test_noalloc_real_energies_match_solver_two_calls(env):
    sb, torch = env
    n, rp, col, val, h = workloads.random_regular(3000, 6, 2, 0.1)
    create = lambda: sb.create_problem_csr(n, rp, col, val, h)  # noqa: E731
    d_rp, d_col = _dev(torch, rp, np.int32), _dev(torch, col, np.int32)
    d_val, d_h = _dev(torch, val, np.float64), _dev(torch, h, np.float64)
    for seed in (5, 6):
        e_ref, _, spins = _solver_energies(sb, create, 8, 4, seed, 120, prec="bf16")
        count = spins.shape[0]
        d_sp = _dev(torch, spins.T, np.int8)
        out = torch.empty(count, dtype=torch.float64, device="cuda")
        sb.energies_csr_noalloc(n, d_rp.data_ptr(), d_col.data_ptr(), d_sp.data_ptr(), count, count,
                                val_f64=d_val.data_ptr(), h_f64=d_h.data_ptr(), energy=out.data_ptr())
        torch.cuda.synchronize()
        assert np.allclose(out.cpu().numpy(), e_ref, rtol=1e-12, atol=1e-9)
        ref = oracle.energies(oracle.Problem.csr(n, rp, col, val, h), spins[:6])
        assert np.allclose(out.cpu().numpy()[:6], ref, rtol=1e-12, atol=1e-9)


def test_noalloc_rejects_sizes_beyond_scratch(env):
    sb, torch = env
    n = 100000  # ceil(n/32) = 3125 row blocks
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    sp = torch.ones((1, 1), dtype=torch.int8, device="cuda")
    out = torch.empty(200, dtype=torch.int64, device="cuda")
    with pytest.raises(sb.SBQAError) as e:
        sb.energies_csr_noalloc(n, rp.data_ptr(), rp.data_ptr(), sp.data_ptr(), 256, 200,
                                val_i32=rp.data_ptr(), energy_int=out.data_ptr())
    assert e.value.status == sb.ERR_UNSUPPORTED
    assert "scratch" in sb.lib.sbqa_last_error().decode()
    with pytest.raises(sb.SBQAError) as e:  # a NULL column array is refused before any launch
        sb.energies_csr_noalloc(8, rp.data_ptr(), 0, sp.data_ptr(), 1, 1,
                                val_i32=rp.data_ptr(), energy_int=out.data_ptr())
    assert e.value.status == sb.ERR_INVALID_ARG
