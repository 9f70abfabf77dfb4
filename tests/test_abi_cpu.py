"""The C-ABI library loads, exports every declared symbol, and rejects bad
input on the host before touching the GPU (CPU only)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sb():
    from paper_2604_01050_gb300 import build as b
    b.build()
    import paper_2604_01050_gb300 as s
    return s


def _declared():
    txt = open(os.path.join(ROOT, "include", "sbqa.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sbqa_[a-z_]+)\s*\(", txt)))


def test_header_declarations_are_exported(sb):
    declared = _declared()
    assert len(declared) >= 15
    lib = ctypes.CDLL(sb.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(sb.EXPORTS) == declared


def test_version_and_strerror(sb):
    assert sb.version() == 100
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert sb.strerror(code) and sb.strerror(code) != "unknown status"
    assert sb.strerror(-99) == "unknown status"


def test_dense_validation_errors_across_row_blocks(sb):
    """The dense checks run per block of 64 rows and per 64 x 64 tile pair:
    errors planted far from the diagonal and in the last, partial block are
    still found (all fail before any device call)."""
    n = 200
    rng = np.random.default_rng(0)
    up = np.triu(rng.choice([-1.0, 1.0], size=(n, n)), 1)
    base = up + up.T
    cases = []
    J = base.copy(); J[3, 190] = -J[3, 190]                       # tile (0, 2) against its mirror
    cases.append((J, None, sb.ERR_NOT_SYMMETRIC))
    J = base.copy(); J[150, 70] += 0.5                            # lower triangle, middle blocks
    cases.append((J, None, sb.ERR_NOT_SYMMETRIC))
    J = base.copy(); J[199, 199] = 1.0                            # diagonal in the partial last block
    cases.append((J, None, sb.ERR_NOT_SYMMETRIC))
    J = base.copy(); J[130, 7] = np.nan; J[7, 130] = np.nan       # NaN
    cases.append((J, None, sb.ERR_NOT_FINITE))
    J = base.copy(); J[66, 65] = np.inf; J[65, 66] = np.inf        # inf at a block edge
    cases.append((J, None, sb.ERR_NOT_FINITE))
    h = np.zeros(n); h[198] = -np.inf
    cases.append((base, h, sb.ERR_NOT_FINITE))
    for J, hh, want in cases:
        with pytest.raises(sb.SBQAError) as e:
            sb.create_problem_dense(J, hh)
        assert e.value.status == want


def test_dense_validation_errors(sb):
    J = np.array([[0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(sb.SBQAError) as e:
        sb.create_problem_dense(np.array([[0.0, 1.0], [2.0, 0.0]]))
    assert e.value.status == sb.ERR_NOT_SYMMETRIC
    with pytest.raises(sb.SBQAError) as e:
        sb.create_problem_dense(np.array([[1.0, 1.0], [1.0, 0.0]]))
    assert e.value.status == sb.ERR_NOT_SYMMETRIC
    with pytest.raises(sb.SBQAError) as e:
        sb.create_problem_dense(np.array([[0.0, np.nan], [np.nan, 0.0]]))
    assert e.value.status == sb.ERR_NOT_FINITE
    with pytest.raises(sb.SBQAError) as e:
        sb.create_problem_dense(J, h=np.array([0.0, np.inf]))
    assert e.value.status == sb.ERR_NOT_FINITE


def test_csr_validation_errors(sb):
    rp = np.array([0, 1, 2]); col = np.array([1, 0]); val = np.array([1.0, 1.0])
    bad = [
        (np.array([0, 1, 3]), col, val, sb.ERR_NOT_SYMMETRIC),          # row_ptr end != nnz
        (rp, np.array([1, 1]), val, sb.ERR_NOT_SYMMETRIC),              # diagonal entry
        (rp, col, np.array([1.0, 2.0]), sb.ERR_NOT_SYMMETRIC),          # asymmetric values
        (rp, np.array([1, 5]), val, sb.ERR_INVALID_ARG),                # column out of range
        (rp, col, np.array([1.0, np.nan]), sb.ERR_NOT_FINITE),
    ]
    for r, c, v, code in bad:
        with pytest.raises(sb.SBQAError) as e:
            sb.create_problem_csr(2, r, c, v)
        assert e.value.status == code
    # unsorted / duplicate columns
    with pytest.raises(sb.SBQAError) as e:
        sb.create_problem_csr(3, [0, 2, 3, 4], [2, 1, 0, 0], [1.0, 1.0, 1.0, 1.0])
    assert e.value.status == sb.ERR_NOT_SYMMETRIC


def test_default_params(sb):
    p = sb.default_params()
    assert (p.a0, p.c0, p.dt, p.gamma0, p.delta_slope, p.init_amp) == (1.0, 0.0, 0.5, 1.0, 0.7, 0.1)
    assert p.jperp_enable == 1 and p.precision == sb.PREC_AUTO and p.eval_every == 0


def test_product_path_has_no_oracle_dependency():
    """The product package never imports, loads or runs the oracle."""
    pkg = os.path.join(ROOT, "paper_2604_01050_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower(), f
