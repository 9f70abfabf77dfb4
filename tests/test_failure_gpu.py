"""Failure detection on the GPU without a fault: a wait that runs out.

The persistent CSR solver's grid barrier is bounded (1 s by %globaltimer).
The host-side test hook SBQA_TEST_SKIP_BARRIER_STEP=n makes block 0 skip its
arrival after step n, so every block's wait runs out; the kernel ends, the
run reports SBQA_ERR_TIMEOUT at the next synchronisation, and the handle
stays usable.  Nothing faults, traps or hangs the device.
"""
import numpy as np
import pytest

import workloads
from sbqa_cases import create, lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as s
    return s


def _solve(sb, spec, kernel_select):
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(8, 1), gamma0=16.0, kernel_select=kernel_select)
    sb.run(prob, 60, 32, 8, seed=1)
    return prob


def test_barrier_timeout_is_reported_and_the_handle_recovers(sb, monkeypatch):
    pb, spec = lattice(8, 3)
    monkeypatch.setenv("SBQA_TEST_SKIP_BARRIER_STEP", "10")
    prob = _solve(sb, spec, 2)
    assert prob.info().step_kernel == 4
    with pytest.raises(sb.SBQAError) as e:
        sb.get_best(prob)
    assert e.value.status == sb.ERR_TIMEOUT
    monkeypatch.delenv("SBQA_TEST_SKIP_BARRIER_STEP")
    sb.run(prob, 60, 32, 8, seed=1)
    xa, _, _ = sb.get_state(prob)
    ea = sb.get_best(prob)["energy"]
    ref = _solve(sb, spec, 1)  # per-step kernels, fresh handle
    xb, _, _ = sb.get_state(ref)
    assert np.array_equal(xa, xb)
    assert np.array_equal(ea, sb.get_best(ref)["energy"])
