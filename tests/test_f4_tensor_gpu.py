"""The persistent dense tensor-core solver with packed e2m1 operands
(tcgen05.mma kind::mxf4 with unit scale factors, J rows resident in shared
memory; step_kernel 15) and its paired form (2-CTA clusters sharing M=256
MMAs, each CTA staging half of every f tile; step_kernel 16).

For integer |J_ij| <= 4 and f in {-1, 0, 1} (Eq. 8) every product and every
partial sum of G = J f is an exact small integer, so the e2m1 solver must
reproduce the e4m3 persistent solver (kernel_select 12, step_kernel 5) bit
for bit: states after whole runs with readouts, split runs and a resume
through set_state.  The e4m3 solvers are tied to the oracle by the per-step
parity tests; here the final energies are also compared with the oracle's
integers of the returned spins.  Shapes cover ragged N (a half-empty last
k-block of 256 spins), ragged R * P, general P and runs wider than 32."""
import numpy as np
import pytest

import oracle
import workloads
from sbqa_cases import create, dense_int, sk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as s
    return s


# name: (oracle problem and spec, P, R)
CASES = {
    "sk2000_P32_R32": (lambda: sk(2000, 3), 32, 32),
    "int4_N300_P8_R16": (lambda: dense_int(300, 5, jmax=4), 8, 16),
    "int3_N1000_P5_R40": (lambda: dense_int(1000, 6, jmax=3), 5, 40),
    "sk700_P64_R4": (lambda: sk(700, 7), 64, 4),
    "int2_N500_P128_R2": (lambda: dense_int(500, 8, jmax=2), 128, 2),
}


def _run(sb, spec, P, R, S, sel, eval_every=13, split=None, seed=4):
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, 3), precision="exact", eval_every=eval_every,
                    kernel_select=sel, gamma0=4.0 * min(P, 32))
    if split is None:
        sb.run(prob, S, P, R, seed=seed)
    else:
        sb.run_begin(prob, S, P, R, seed=seed)
        sb.run_advance(prob, split)
        sb.run_advance(prob, S)
        sb.run_finish(prob)
    return prob


def _pairs(N):
    """The paired form takes padded N a multiple of 256."""
    return -(-N // 128) * 128 % 256 == 0


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("sel", [15, 14])
def test_e2m1_solver_equals_e4m3_persistent(sb, name, sel):
    make, P, R = CASES[name]
    pb, spec = make()
    S = 60
    ref = _run(sb, spec, P, R, S, 12)
    assert ref.info().step_kernel == 5
    xr, yr, _ = sb.get_state(ref)
    want = 16 if sel == 14 and _pairs(pb.n) else 15
    got = _run(sb, spec, P, R, S, sel)
    assert got.info().step_kernel == want
    xg, yg, _ = sb.get_state(got)
    assert np.array_equal(xg, xr) and np.array_equal(yg, yr)
    assert np.array_equal(sb.get_best(got)["energy"], sb.get_best(ref)["energy"])
    _, ei = sb.get_energies(got)
    spins = np.where(xg >= 0, 1, -1).astype(np.int8)
    assert np.array_equal(ei, oracle.energies(pb, spins))
    split = _run(sb, spec, P, R, S, sel, split=23)
    assert split.info().step_kernel == want
    xs, ys, _ = sb.get_state(split)
    assert np.array_equal(xs, xr) and np.array_equal(ys, yr)


@pytest.mark.parametrize("N,sel,want", [(600, 14, 15), (1000, 14, 16), (1000, 15, 15)])
def test_e2m1_solver_resume_through_set_state(sb, N, sel, want):
    """set_state rebuilds the packed f buffer from the state: a run resumed
    from a dumped mid-run state equals the unbroken run bit for bit."""
    pb, spec = dense_int(N, 11, jmax=4)
    P, R, S = 16, 16, 80
    prob = create(sb, spec)
    sb.set_schedule(prob, *workloads.autotune_params(R, 5), precision="exact", kernel_select=sel, gamma0=32.0)
    sb.run_begin(prob, S, P, R, seed=9)
    sb.run_advance(prob, 31)
    x31, y31, _ = sb.get_state(prob)
    sb.run_advance(prob, S)
    xa, ya, _ = sb.get_state(prob)
    assert prob.info().step_kernel == want
    sb.run_begin(prob, S, P, R, seed=1234)
    sb.set_state(prob, x31, y31, 31)
    sb.run_advance(prob, S)
    xb, yb, _ = sb.get_state(prob)
    assert np.array_equal(xa, xb) and np.array_equal(ya, yb)


def test_e2m1_solver_not_taken_beyond_its_range(sb):
    """|J_ij| = 5 has no e2m1 value, and padded N = 2432 leaves no room for the
    resident J rows: kernel_select 14 then runs the e4m3 persistent solver."""
    _, spec = dense_int(400, 12, jmax=5)
    prob = _run(sb, spec, 8, 16, 20, 14)
    assert prob.info().step_kernel == 5
    _, spec = sk(2400, 13)
    prob = _run(sb, spec, 8, 16, 10, 14, eval_every=0)
    assert prob.info().step_kernel == 5


def test_autotuner_times_the_e2m1_solver(sb):
    """With kernel_select 0 the autotuner times the e2m1 solver beside the
    others; whichever it keeps, the result equals the e4m3 solver's."""
    pb, spec = sk(2000, 14)
    P, R, S = 32, 32, 40
    auto = _run(sb, spec, P, R, S, 0)
    info = auto.info()
    print("autotuner: step_kernel %d, persistent %.2f us/step" % (info.step_kernel, 1e3 * info.persistent_ms))
    assert info.step_kernel in (2, 5, 8, 9, 15, 16)
    ref = _run(sb, spec, P, R, S, 12)
    assert np.array_equal(sb.get_state(auto)[0], sb.get_state(ref)[0])
