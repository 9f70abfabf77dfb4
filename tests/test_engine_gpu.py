"""The batching engine: mixed requests (sparse +-1, sparse BF16, dense on the
tensor cores, dense on CUDA cores, ragged shapes) give exactly the result of
solving each alone with sbqa_run, whatever the mix, the chunk size and the
admission order."""
import numpy as np
import pytest

import oracle
import workloads
from sbqa_cases import create, dense_int, dense_real, lattice, regular, sk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sb():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as s
    return s


def _sk_real_h(n, seed):
    """+-1 SK couplings with a Gaussian field: the product is exact on the
    tensor cores, the energies are not integers."""
    J, _ = workloads.sk_pm1(n, seed)
    return ("dense", J, np.random.default_rng(seed).normal(0.0, 0.5, n))


def _requests(sb, with_oracle=False):
    """(problem handle, steps, P, R, seed) of a mixed workload (and the oracle's
    problem of each, with_oracle=True)."""
    out, orc = [], []
    for k, (spec, steps, P, R, prec) in enumerate([
            (lattice(8, 1)[1], 90, 8, 4, "auto"),
            (regular(500, 6, 3)[1], 130, 16, 2, "bf16"),
            (sk(300, 2)[1], 70, 8, 3, "exact"),       # tcgen05 FP8 path
            (sk(100, 5)[1], 100, 4, 5, "auto"),       # dense CUDA-core path
            (lattice(5, 2)[1], 50, 2, 3, "auto"),     # ragged columns
            (dense_int(260, 7, jmax=2)[1], 64, 32, 2, "exact"),
            (lattice(7, 4)[1], 60, 2, 99, "auto"),    # 8 columns per lane, ragged inside a lane (R P = 198)
            (regular(400, 6, 5)[1], 80, 16, 16, "bf16"),  # 8 columns per lane, ELL values
            (lattice(6, 6)[1], 40, 2, 201, "auto"),   # 8 columns per lane, ragged inside a lane (R P = 402)
            (regular(300, 6, 7)[1], 40, 32, 16, "fp32"),  # 8 columns per lane, FP32 ELL values, R P = 512
            (_sk_real_h(300, 9), 50, 8, 2, "auto"),   # tcgen05 product, FP64 readout (non-integer h)
    ]):
        pb = create(sb, spec)
        sb.set_schedule(pb, *workloads.autotune_params(R, k), precision=prec, eval_every=0)
        out.append((pb, steps, P, R, 100 + k))
        if with_oracle:
            orc.append(oracle.Problem.dense(spec[1], spec[2]) if spec[0] == "dense"
                       else oracle.Problem.csr(*spec[1:]))
    return (out, orc) if with_oracle else out


def _alone(sb, req):
    pb, steps, P, R, seed = req
    sb.run(pb, steps, P, R, seed=seed)
    return sb.get_best(pb)


@pytest.mark.parametrize("chunk,slots,arena_mb", [(32, 16, 512), (7, 3, 512), (50, 16, 40)])
def test_engine_mix_equals_alone(sb, chunk, slots, arena_mb):
    reqs, orcs = _requests(sb, with_oracle=True)
    alone = [_alone(sb, r) for r in reqs]
    eng = sb.engine_create(arena_mb << 20, slots, chunk)
    ids = [sb.engine_submit(eng, *r) for r in reqs]
    done = []
    for _ in range(10000):
        done += sb.engine_step(eng)
        st = sb.engine_stats(eng)
        assert st["active"] <= slots and st["arena_used"] <= st["arena_bytes"]
        if len(done) == len(ids):
            break
    assert sorted(done) == ids
    for rid, ref, pbo in zip(ids, alone, orcs):
        got = sb.engine_result(eng, rid)
        assert np.array_equal(got["spins"], ref["spins"]), rid
        assert np.array_equal(got["energy"], ref["energy"]), rid
        assert np.array_equal(got["replica"], ref["replica"]), rid
        # and directly against the oracle: the energies of the returned spins
        e_o = oracle.energies(pbo, got["spins"])
        if pbo.is_integer:
            assert np.array_equal(got["energy_int"], e_o), rid
        else:
            assert np.allclose(got["energy"], e_o, rtol=1e-12, atol=1e-9), rid
    st = sb.engine_stats(eng)
    assert st["finished"] == len(ids) and st["queued"] == 0 and st["active"] == 0 and st["arena_used"] == 0


def test_engine_batches_small_dense_requests(sb):
    """Small dense tensor-core requests share cooperative launches: e4m3 and
    BF16 operands, run widths 8 and 16, a ring of 6 replicas in 8 columns,
    step counts that end inside a chunk, and more tiles of one form than one
    wave holds (two launches for that form).  Every result equals the request
    solved alone."""
    reqs, orcs = [], []
    for k in range(17):
        if k < 11:
            (pbo, spec), prec, P, R = sk(1000, 40 + k), "exact", 16, 16     # 8 x 2 = 16 tiles each
        elif k < 14:
            (pbo, spec), prec, P, R = dense_real(300, 40 + k), "bf16", 8, 4  # BF16 operands, 3 x 1 tiles
        else:
            (pbo, spec), prec, P, R = dense_int(200, 40 + k, jmax=3), "exact", 6, 5  # ring of 6 in 8 columns
        orcs.append(pbo)
        pb = create(sb, spec)
        sb.set_schedule(pb, *workloads.autotune_params(R, k), precision=prec, eval_every=0)
        reqs.append((pb, 40 + 7 * k, P, R, 300 + k))
    alone = [_alone(sb, r) for r in reqs]
    for batching in (True, False):
        eng = sb.engine_create(2 << 30, 32, 25)
        sb.engine_set_dense_batching(eng, batching)
        ids = [sb.engine_submit(eng, *r) for r in reqs]
        done = []
        for _ in range(1000):
            done += sb.engine_step(eng)
            if len(done) == len(ids):
                break
        assert sorted(done) == ids
        for rid, ref, pbo in zip(ids, alone, orcs):
            got = sb.engine_result(eng, rid)
            assert np.array_equal(got["spins"], ref["spins"]), (batching, rid)
            assert np.array_equal(got["energy"], ref["energy"]), (batching, rid)
            assert np.array_equal(got["replica"], ref["replica"]), (batching, rid)
            e_o = oracle.energies(pbo, got["spins"])
            if pbo.is_integer:
                assert np.array_equal(got["energy_int"], e_o), (batching, rid)
            else:
                assert np.allclose(got["energy"], e_o, rtol=1e-12, atol=1e-9), (batching, rid)
        st = sb.engine_stats(eng)
        assert st["dense_e2m1_requests"] == 11  # the +-1 requests (N=200 stays below the tensor cores)
        if batching:
            # the first chunk alone needs two launches of the 16-tile form (176 tiles), one of each other form
            assert st["dense_batched_launches"] >= 4
            assert st["dense_batched_chunks"] >= 2 * st["dense_batched_launches"]
        else:
            assert st["dense_batched_launches"] == 0 and st["dense_batched_chunks"] == 0
        eng.destroy()
    with pytest.raises(sb.SBQAError) as e:
        sb.engine_set_dense_batching(sb.engine_create(64 << 20, 2, 10), 2)
    assert e.value.status == sb.ERR_INVALID_ARG


def test_engine_e2m1_and_e4m3_requests_agree(sb):
    """Dense requests with integer |J| <= 4 run on the e2m1 solver in the
    engine -- batched, or alone when their tiles fill most of the device (SK
    N=2000, R*P=1024: 128 tiles) -- and with kernel_select 12 on the e4m3
    solvers; both give the same spins and the oracle's energies of them."""
    specs = [(sk(700, 60), 16, 8), (dense_int(300, 61, jmax=4), 8, 16), (sk(2000, 62), 32, 32),
             (dense_int(500, 63, jmax=2), 5, 24)]
    results = {}
    for sel in (0, 12):
        eng = sb.engine_create(2 << 30, 8, 30)
        ids = []
        for k, ((pbo, spec), P, R) in enumerate(specs):
            pb = create(sb, spec)
            sb.set_schedule(pb, *workloads.autotune_params(R, k), precision="exact", eval_every=0,
                            kernel_select=sel)
            ids.append(sb.engine_submit(eng, pb, 75, P, R, seed=500 + k))
        done = []
        for _ in range(1000):
            done += sb.engine_step(eng)
            if len(done) == len(ids):
                break
        assert sorted(done) == ids
        results[sel] = [sb.engine_result(eng, i) for i in ids]
        assert sb.engine_stats(eng)["dense_e2m1_requests"] == (len(specs) if sel == 0 else 0)
        eng.destroy()
    for a, b, ((pbo, _), _, _) in zip(results[0], results[12], specs):
        assert np.array_equal(a["spins"], b["spins"]) and np.array_equal(a["energy_int"], b["energy_int"])
        assert np.array_equal(a["energy_int"], oracle.energies(pbo, a["spins"]))


def test_engine_admission_waits_for_memory(sb):
    """An arena that holds one lattice request at a time runs them one after another."""
    n, rp, col, val, h = workloads.cubic_lattice(10, 0)
    pb = sb.create_problem_csr(n, rp, col, val, h)
    sb.set_schedule(pb, *workloads.autotune_params(8, 0))
    one = 1000 * 8 * 4 * 11 + (8 << 20) // 8  # about one request's state
    eng = sb.engine_create(max(one, 1 << 20) * 2, 8, 25)
    ids = [sb.engine_submit(eng, pb, 60, 16, 8, seed=s) for s in range(3)]
    order = []
    while len(order) < 3:
        order += sb.engine_step(eng)
        assert sb.engine_stats(eng)["active"] <= 2
    assert sorted(order) == ids
    for rid, s in zip(ids, range(3)):
        sb.run(pb, 60, 16, 8, seed=s)
        assert np.array_equal(sb.engine_result(eng, rid)["energy"], sb.get_best(pb)["energy"])


def test_engine_rejects_bad_requests(sb):
    pb, spec = sk(32, 0)
    prob = create(sb, spec)
    eng = sb.engine_create(64 << 20, 4, 10)
    with pytest.raises(sb.SBQAError) as e:
        sb.engine_submit(eng, prob, 10, 8, 2)
    assert e.value.status == sb.ERR_STATE  # no schedule yet
    sb.set_schedule(prob)
    with pytest.raises(sb.SBQAError) as e:
        sb.engine_submit(eng, prob, 10, 200, 2)  # more than 128 replicas per run
    assert e.value.status == sb.ERR_UNSUPPORTED
    with pytest.raises(sb.SBQAError) as e:
        sb.engine_result(eng, 0)
    assert e.value.status == sb.ERR_INVALID_ARG
    sb.set_schedule(prob, variant="ballistic")  # served by sbqa_run, not by the engine
    with pytest.raises(sb.SBQAError) as e:
        sb.engine_submit(eng, prob, 10, 8, 2)
    assert e.value.status == sb.ERR_UNSUPPORTED
    with pytest.raises(sb.SBQAError) as e:
        sb.set_schedule(prob, variant=2)
    assert e.value.status == sb.ERR_INVALID_ARG
