"""Failure detection on the GPU without a fault: a wait that runs out.

The persistent CSR solver's grid barrier is bounded (1 s by %globaltimer).
The host-side test hook SBQA_TEST_SKIP_BARRIER_STEP=n makes block 0 skip its
arrival after step n, so every block's wait runs out; the kernel ends, the
run reports SBQA_ERR_TIMEOUT at the next synchronisation, and the handle
stays usable.  The batching engine's host hook
SBQA_TEST_ENGINE_FAIL_REQUEST=id makes it read one request's device error
word as set: that request is retired with TIMEOUT and the others complete.
With SBQA_TEST_ENGINE_HOLD_DENSE=id one dense request of a batched
tensor-core launch leaves a step counter unpublished, so the waits of its
own tiles run out on the device (2 s) while the other requests of the same
launch complete.  Nothing faults, traps or hangs the device.
"""
import numpy as np
import pytest

import workloads
from sbqa_cases import create, lattice, sk

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


def test_engine_retires_a_failed_request_and_keeps_serving(sb, monkeypatch):
    """A request whose device wait gave up (the host hook SBQA_TEST_ENGINE_FAIL_REQUEST=id makes the
    engine read that request's error word as set) is retired with TIMEOUT: its slot and arena space are
    released, the requests beside it and after it complete with the result of solving them alone."""
    specs = [lattice(6, 1)[1], lattice(5, 2)[1], lattice(6, 3)[1], lattice(5, 4)[1]]
    probs = []
    for k, spec in enumerate(specs):
        pb = create(sb, spec)
        sb.set_schedule(pb, *workloads.autotune_params(4, k), eval_every=0)
        probs.append(pb)
    eng = sb.engine_create(256 << 20, 2, 20)  # two slots: the last two requests wait for the first two
    ids = [sb.engine_submit(eng, pb, 40, 8, 4, seed=10 + k) for k, pb in enumerate(probs)]
    monkeypatch.setenv("SBQA_TEST_ENGINE_FAIL_REQUEST", str(ids[1]))
    done, timeouts = [], 0
    for _ in range(100):
        try:
            done += sb.engine_step(eng)
        except sb.SBQAError as e:
            assert e.status == sb.ERR_TIMEOUT
            timeouts += 1
            done += e.done_ids
        if len(done) == len(ids):
            break
    assert sorted(done) == ids and timeouts == 1
    with pytest.raises(sb.SBQAError) as e:
        sb.engine_result(eng, ids[1])
    assert e.value.status == sb.ERR_TIMEOUT
    for k in (0, 2, 3):
        sb.run(probs[k], 40, 8, 4, seed=10 + k)
        assert np.array_equal(sb.engine_result(eng, ids[k])["energy"], sb.get_best(probs[k])["energy"])
    st = sb.engine_stats(eng)
    assert st["active"] == 0 and st["arena_used"] == 0 and st["finished"] == 4


def test_engine_dense_batch_isolates_a_request_whose_wait_runs_out(sb, monkeypatch):
    """Three dense tensor-core requests share each chunk's batched launch.  The
    middle one's tile (0, 0) never publishes its step counter (host hook
    SBQA_TEST_ENGINE_HOLD_DENSE=id), so the bounded waits of that request's
    tiles run out on the device and it is retired with TIMEOUT; the other two
    requests of the same launches complete with the results of solving them
    alone."""
    probs = []
    for k in range(3):
        pb = create(sb, sk(300, 30 + k)[1])
        sb.set_schedule(pb, *workloads.autotune_params(4, k), precision="exact", eval_every=0)
        probs.append(pb)
    eng = sb.engine_create(512 << 20, 8, 25)
    ids = [sb.engine_submit(eng, pb, 60, 8, 4, seed=40 + k) for k, pb in enumerate(probs)]
    monkeypatch.setenv("SBQA_TEST_ENGINE_HOLD_DENSE", str(ids[1]))
    done, timeouts = [], 0
    for _ in range(100):
        try:
            done += sb.engine_step(eng)
        except sb.SBQAError as e:
            assert e.status == sb.ERR_TIMEOUT
            timeouts += 1
            done += e.done_ids
        if len(done) == len(ids):
            break
    monkeypatch.delenv("SBQA_TEST_ENGINE_HOLD_DENSE")
    assert sorted(done) == ids and timeouts == 1
    with pytest.raises(sb.SBQAError) as e:
        sb.engine_result(eng, ids[1])
    assert e.value.status == sb.ERR_TIMEOUT
    st = sb.engine_stats(eng)
    assert st["dense_batched_launches"] >= 1 and st["dense_batched_chunks"] >= 2 * st["dense_batched_launches"]
    for k in (0, 2):
        sb.run(probs[k], 60, 8, 4, seed=40 + k)
        ref = sb.get_best(probs[k])
        got = sb.engine_result(eng, ids[k])
        assert np.array_equal(got["energy"], ref["energy"]) and np.array_equal(got["spins"], ref["spins"])
    # the engine keeps serving: a new request on the failed one's problem completes
    rid = sb.engine_submit(eng, probs[1], 60, 8, 4, seed=41)
    done = []
    for _ in range(100):
        done += sb.engine_step(eng)
        if rid in done:
            break
    sb.run(probs[1], 60, 8, 4, seed=41)
    assert np.array_equal(sb.engine_result(eng, rid)["energy"], sb.get_best(probs[1])["energy"])
