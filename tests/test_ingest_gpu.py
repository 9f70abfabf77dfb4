"""Dense J read by the GPU from the caller's array (N >= 1024): the same
checks, errors and analysis as the host pass, bit-identical solves on every
path the library takes from its device copy (e4m3 and bfloat16 tensor-core
operands, the CUDA-core FP32 / bfloat16 copies, int32 and FP64 readout
values), and the oracle's energies on the spins it returns.  The host pass
is forced with the test hook SBQA_TEST_HOST_INGEST=1."""
import os

import numpy as np
import pytest

import oracle
import workloads
from sbqa_cases import dense_int, dense_real

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as s
    return s


def _create(sb, J, h, host):
    if host:
        os.environ["SBQA_TEST_HOST_INGEST"] = "1"
    try:
        return sb.create_problem_dense(J, h)
    finally:
        os.environ.pop("SBQA_TEST_HOST_INGEST", None)


def _sk(n, seed, real_h=False):
    J, _ = workloads.sk_pm1(n, seed)
    h = np.random.default_rng(seed).normal(0.0, 0.5, n) if real_h else None
    return J, h


# name, (J, h), precisions run on both handles
CASES = {
    "pm1": (lambda: _sk(1100, 5), ("auto", "fp32", "bf16")),        # e4m3 operands, int32 readout
    "pm1_real_h": (lambda: _sk(1030, 6, True), ("auto", "fp32")),     # integer J beside a real h: FP64 readout
    "int3": (lambda: dense_int(1050, 7, jmax=3)[1][1:], ("auto", "fp32")),
    "int200": (lambda: dense_int(1090, 8, jmax=200)[1][1:], ("auto", "bf16")),  # |J| > 127: FP64 copy, exact BF16
    "real": (lambda: dense_real(1040, 9, 0.3)[1][1:], ("bf16", "fp32")),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_device_ingest_equals_host_pass(sb, name):
    make, precs = CASES[name]
    J, h = make()
    pd = _create(sb, J, h, host=False)
    ph = _create(sb, J, h, host=True)
    idv, ihs = pd.info(), ph.info()
    assert idv.j_on_device == 1 and ihs.j_on_device == 0
    for f in ("n", "is_dense", "nnz", "is_integer", "max_abs_j"):
        assert getattr(idv, f) == getattr(ihs, f), f
    # the sum of squares is added in another order (per row on the device, per
    # 64-row block on the host): equal for integer J, to rounding otherwise
    # (N^2 ~ 10^6 terms: a relative bound of 10^-12 is far above their rounding)
    assert abs(idv.c0_auto - ihs.c0_auto) <= 1e-12 * ihs.c0_auto
    if idv.is_integer:
        assert idv.c0_auto == ihs.c0_auto
    pb_o = oracle.Problem.dense(J, h)
    beta, alpha = workloads.autotune_params(4, 1)
    for prec in precs:
        for pb in (pd, ph):
            sb.set_schedule(pb, beta, alpha, precision=prec, c0=ihs.c0_auto, eval_every=20)
            sb.run(pb, 60, 8, 4, seed=11)
        assert pd.info().step_kernel == ph.info().step_kernel, prec
        sd, sh = sb.get_state(pd), sb.get_state(ph)
        assert np.array_equal(sd[0], sh[0]) and np.array_equal(sd[1], sh[1]), prec
        bd, bh = sb.get_best(pd), sb.get_best(ph)
        assert np.array_equal(bd["spins"], bh["spins"]) and np.array_equal(bd["energy"], bh["energy"]), prec
        ref = oracle.energies(pb_o, bd["spins"])
        if pb_o.is_integer:
            assert np.array_equal(bd["energy_int"], ref), prec
        else:
            assert np.allclose(bd["energy"], ref, rtol=1e-12, atol=1e-9), prec


def test_device_ingest_rejects_what_the_host_pass_rejects(sb):
    J, _ = workloads.sk_pm1(1060, 3)
    bad = []
    A = J.copy(); A[3, 700] += 1.0                      # J != J^T, far from the diagonal tiles
    bad.append((A, None, sb.ERR_NOT_SYMMETRIC))
    B = J.copy(); B[1059, 1058] = 2.0                    # ragged last tile
    bad.append((B, None, sb.ERR_NOT_SYMMETRIC))
    D = J.copy(); D[5, 5] = 1.0                          # nonzero diagonal
    bad.append((D, None, sb.ERR_NOT_SYMMETRIC))
    F = J.copy(); F[10, 20] = F[20, 10] = np.nan
    bad.append((F, None, sb.ERR_NOT_FINITE))
    G = J.copy(); G[30, 31] = G[31, 30] = np.inf
    bad.append((G, None, sb.ERR_NOT_FINITE))
    hh = np.zeros(1060); hh[7] = np.inf
    bad.append((J, hh, sb.ERR_NOT_FINITE))
    for M, h, code in bad:
        for host in (False, True):
            with pytest.raises(sb.SBQAError) as e:
                _create(sb, M, h, host)
            assert e.value.status == code, (host, code)
    # and the clean matrix is accepted by both
    assert _create(sb, J, None, False).info().j_on_device == 1
