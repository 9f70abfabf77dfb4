"""ctypes binding of the C ABI in include/sbqa.h (argument marshalling only).

Every function keeps the C name without the ``sbqa_`` prefix.  Arrays are
numpy arrays in host memory; ``stream`` is a raw ``cudaStream_t`` value (an
int) or any object with a ``cuda_stream`` attribute (a torch.cuda.Stream).
Failures raise :class:`SBQAError` with the status code and the library's
detail message.  There is no fallback: if ``libsbqa.so`` is missing the
import fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsbqa.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_NOT_SYMMETRIC = -2
ERR_NOT_FINITE = -3
ERR_OOM = -4
ERR_CUDA = -5
ERR_STATE = -6
ERR_UNSUPPORTED = -7
ERR_TIMEOUT = -8

PREC_AUTO, PREC_FP32, PREC_EXACT, PREC_BF16 = 0, 1, 2, 3
PRECISIONS = {"auto": PREC_AUTO, "fp32": PREC_FP32, "exact": PREC_EXACT, "bf16": PREC_BF16}
VARIANT_THRESHOLD = 0
VARIANT_BALLISTIC = 1
VARIANTS = {"threshold": VARIANT_THRESHOLD, "ballistic": VARIANT_BALLISTIC}

# Every symbol include/sbqa.h declares.
EXPORTS = (
    "sbqa_create_problem_dense", "sbqa_create_problem_csr", "sbqa_destroy", "sbqa_release_cached_memory",
    "sbqa_get_problem_info", "sbqa_default_params", "sbqa_set_schedule", "sbqa_run",
    "sbqa_run_begin", "sbqa_run_advance", "sbqa_run_finish", "sbqa_synchronize",
    "sbqa_get_best", "sbqa_get_energies", "sbqa_get_state", "sbqa_set_state",
    "sbqa_strerror", "sbqa_last_error", "sbqa_version", "sbqa_energies_csr_noalloc",
    "sbqa_engine_create", "sbqa_engine_destroy", "sbqa_engine_submit", "sbqa_engine_step",
    "sbqa_engine_result", "sbqa_engine_stats", "sbqa_engine_set_dense_batching",
)


class SBQAError(RuntimeError):
    def __init__(self, status, func, detail):
        super().__init__("%s failed: %s (%d): %s" % (func, strerror(status), status, detail))
        self.status = status


class ProblemInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("is_dense", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("is_integer", ctypes.c_int32), ("max_abs_j", ctypes.c_int32),
                ("c0_auto", ctypes.c_double), ("step_kernel", ctypes.c_int32),
                ("step_variant", ctypes.c_int32), ("variant_ms", ctypes.c_float * 8),
                ("persistent_ms", ctypes.c_float), ("j_on_device", ctypes.c_int32)]


class EngineStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int32), ("active", ctypes.c_int32), ("finished", ctypes.c_int32),
                ("arena_bytes", ctypes.c_int64), ("arena_used", ctypes.c_int64),
                ("updates_issued", ctypes.c_int64), ("kernels_launched", ctypes.c_int64),
                ("batched_updates", ctypes.c_int64), ("batched_ms", ctypes.c_double),
                ("dense_batched_launches", ctypes.c_int64), ("dense_batched_chunks", ctypes.c_int64),
                ("dense_e2m1_requests", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("c0", ctypes.c_double), ("dt", ctypes.c_double),
                ("gamma0", ctypes.c_double), ("delta_slope", ctypes.c_double),
                ("init_amp", ctypes.c_double), ("jperp_enable", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("eval_every", ctypes.c_int32), ("n_runs", ctypes.c_int32),
                ("kernel_select", ctypes.c_int32), ("beta", ctypes.POINTER(ctypes.c_double)),
                ("alpha", ctypes.POINTER(ctypes.c_double))]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsbqa.so is not built (%s); run paper_2604_01050_gb300.build.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sig = {
        "sbqa_create_problem_dense": (ctypes.c_int, [i32, P(dbl), P(dbl), P(vp)]),
        "sbqa_create_problem_csr": (ctypes.c_int, [i32, i64, P(i64), P(i32), P(dbl), P(dbl), P(vp)]),
        "sbqa_destroy": (None, [vp]),
        "sbqa_release_cached_memory": (ctypes.c_int, []),
        "sbqa_get_problem_info": (ctypes.c_int, [vp, P(ProblemInfo)]),
        "sbqa_default_params": (None, [P(Params)]),
        "sbqa_set_schedule": (ctypes.c_int, [vp, P(Params)]),
        "sbqa_run": (ctypes.c_int, [vp, i32, i32, i32, u64, vp]),
        "sbqa_run_begin": (ctypes.c_int, [vp, i32, i32, i32, u64, vp]),
        "sbqa_run_advance": (ctypes.c_int, [vp, i32]),
        "sbqa_run_finish": (ctypes.c_int, [vp]),
        "sbqa_synchronize": (ctypes.c_int, [vp]),
        "sbqa_get_best": (ctypes.c_int, [vp, P(ctypes.c_int8), P(dbl), P(i64), P(i32), P(i32)]),
        "sbqa_get_energies": (ctypes.c_int, [vp, P(dbl), P(i64)]),
        "sbqa_get_state": (ctypes.c_int, [vp, P(ctypes.c_float), P(ctypes.c_float), P(i32)]),
        "sbqa_set_state": (ctypes.c_int, [vp, P(ctypes.c_float), P(ctypes.c_float), i32]),
        "sbqa_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "sbqa_last_error": (ctypes.c_char_p, []),
        "sbqa_version": (ctypes.c_int, []),
        "sbqa_energies_csr_noalloc": (ctypes.c_int, [i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp]),
        "sbqa_engine_create": (ctypes.c_int, [i64, i32, i32, P(vp)]),
        "sbqa_engine_destroy": (None, [vp]),
        "sbqa_engine_submit": (ctypes.c_int, [vp, vp, i32, i32, i32, u64, P(i32)]),
        "sbqa_engine_step": (ctypes.c_int, [vp, vp, P(i32), P(i32), i32]),
        "sbqa_engine_result": (ctypes.c_int, [vp, i32, P(ctypes.c_int8), P(dbl), P(i64), P(i32)]),
        "sbqa_engine_stats": (ctypes.c_int, [vp, P(EngineStats)]),
        "sbqa_engine_set_dense_batching": (ctypes.c_int, [vp, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def strerror(status: int) -> str:
    return lib.sbqa_strerror(int(status)).decode()


def _check(status, func):
    if status != OK:
        raise SBQAError(status, func, lib.sbqa_last_error().decode())


def _p(a, ctype):
    if a is None:
        return ctypes.cast(None, ctypes.POINTER(ctype))
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


def version() -> int:
    return int(lib.sbqa_version())


def release_cached_memory() -> None:
    """Return the device blocks the library keeps from destroyed problems to the driver."""
    _check(lib.sbqa_release_cached_memory(), "release_cached_memory")


def default_params() -> Params:
    p = Params()
    lib.sbqa_default_params(ctypes.byref(p))
    return p


class Problem:
    """Owning wrapper of one ``sbqa_problem*`` handle."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        self._keep = []
        self.R = self.P = 0

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.sbqa_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    @property
    def handle(self):
        return self._h

    @property
    def n(self):
        return self.info().n

    def info(self) -> ProblemInfo:
        inf = ProblemInfo()
        _check(lib.sbqa_get_problem_info(self._h, ctypes.byref(inf)), "get_problem_info")
        return inf


def create_problem_dense(J, h=None) -> Problem:
    J = np.ascontiguousarray(J, dtype=np.float64)
    n = J.shape[0]
    if J.shape != (n, n):
        raise ValueError("J must be square")
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib.sbqa_create_problem_dense(n, _p(J, ctypes.c_double), _p(hh, ctypes.c_double),
                                         ctypes.byref(out)), "create_problem_dense")
    return Problem(out.value)


def create_problem_csr(n, row_ptr, col_idx, val, h=None) -> Problem:
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    va = np.ascontiguousarray(val, dtype=np.float64)
    hh = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
    out = ctypes.c_void_p()
    _check(lib.sbqa_create_problem_csr(int(n), int(ci.size), _p(rp, ctypes.c_int64), _p(ci, ctypes.c_int32),
                                       _p(va, ctypes.c_double), _p(hh, ctypes.c_double), ctypes.byref(out)),
           "create_problem_csr")
    return Problem(out.value)


def set_schedule(pb: Problem, beta=None, alpha=None, **kw):
    """Keyword names follow ``sbqa_params``; ``precision`` may be a name
    ('auto', 'fp32', 'exact', 'bf16'), ``variant`` 'threshold' or 'ballistic'."""
    prm = default_params()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        if k == "jperp_enable":
            v = int(bool(v))
        setattr(prm, k, v)
    if beta is not None:
        b = np.ascontiguousarray(beta, dtype=np.float64)
        a = np.ascontiguousarray(alpha, dtype=np.float64)
        prm.n_runs = b.size
        prm.beta = _p(b, ctypes.c_double)
        prm.alpha = _p(a, ctypes.c_double)
    _check(lib.sbqa_set_schedule(pb.handle, ctypes.byref(prm)), "set_schedule")


def run(pb: Problem, steps, P, R, seed=0, stream=None):
    _check(lib.sbqa_run(pb.handle, int(steps), int(P), int(R), ctypes.c_uint64(seed), _stream(stream)), "run")
    pb.P, pb.R = int(P), int(R)


def run_begin(pb: Problem, steps, P, R, seed=0, stream=None):
    _check(lib.sbqa_run_begin(pb.handle, int(steps), int(P), int(R), ctypes.c_uint64(seed), _stream(stream)),
           "run_begin")
    pb.P, pb.R = int(P), int(R)


def run_advance(pb: Problem, n_steps):
    _check(lib.sbqa_run_advance(pb.handle, int(n_steps)), "run_advance")


def run_finish(pb: Problem):
    _check(lib.sbqa_run_finish(pb.handle), "run_finish")


def synchronize(pb: Problem):
    _check(lib.sbqa_synchronize(pb.handle), "synchronize")


def get_best(pb: Problem):
    R, N = pb.R, pb.n
    spins = np.empty((R, N), dtype=np.int8)
    e = np.empty(R)
    ei = np.zeros(R, dtype=np.int64)
    k = np.empty(R, dtype=np.int32)
    st = np.empty(R, dtype=np.int32)
    _check(lib.sbqa_get_best(pb.handle, _p(spins, ctypes.c_int8), _p(e, ctypes.c_double), _p(ei, ctypes.c_int64),
                             _p(k, ctypes.c_int32), _p(st, ctypes.c_int32)), "get_best")
    return {"spins": spins, "energy": e, "energy_int": ei, "replica": k, "step": st}


def get_energies(pb: Problem):
    e = np.empty((pb.R, pb.P))
    ei = np.zeros((pb.R, pb.P), dtype=np.int64)
    _check(lib.sbqa_get_energies(pb.handle, _p(e, ctypes.c_double), _p(ei, ctypes.c_int64)), "get_energies")
    return e, ei


def get_state(pb: Problem):
    x = np.empty((pb.R, pb.P, pb.n), dtype=np.float32)
    y = np.empty_like(x)
    sd = ctypes.c_int32()
    _check(lib.sbqa_get_state(pb.handle, _p(x, ctypes.c_float), _p(y, ctypes.c_float), ctypes.byref(sd)),
           "get_state")
    return x, y, sd.value


def set_state(pb: Problem, x, y, step_done):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    _check(lib.sbqa_set_state(pb.handle, _p(x, ctypes.c_float), _p(y, ctypes.c_float), int(step_done)),
           "set_state")


def energies_csr_noalloc(n, row_ptr, col_idx, spins, ld, count, val_i32=0, val_f64=0, h_i64=0, h_f64=0,
                         energy_int=0, energy=0, stream=None):
    """Energies of ``count`` spin configurations with no device allocation.

    Every array argument is a device address (an int, e.g. ``tensor.data_ptr()``;
    0 for NULL); see sbqa_energies_csr_noalloc in include/sbqa.h."""
    _check(lib.sbqa_energies_csr_noalloc(int(n), row_ptr, col_idx, val_i32 or None, val_f64 or None,
                                         h_i64 or None, h_f64 or None, spins, int(ld), int(count),
                                         energy_int or None, energy or None, _stream(stream) or None),
           "energies_csr_noalloc")


class Engine:
    """Owning wrapper of one ``sbqa_engine*`` (continuous batching)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        self.requests = {}  # id -> (problem, R, N)

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.sbqa_engine_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    @property
    def handle(self):
        return self._h


def engine_create(arena_bytes, max_slots, chunk_steps) -> Engine:
    out = ctypes.c_void_p()
    _check(lib.sbqa_engine_create(int(arena_bytes), int(max_slots), int(chunk_steps), ctypes.byref(out)),
           "engine_create")
    return Engine(out.value)


def engine_set_dense_batching(eng: Engine, on: bool):
    _check(lib.sbqa_engine_set_dense_batching(eng.handle, int(on)), "engine_set_dense_batching")


def engine_submit(eng: Engine, pb: Problem, steps, P, R, seed=0) -> int:
    rid = ctypes.c_int32()
    _check(lib.sbqa_engine_submit(eng.handle, pb.handle, int(steps), int(P), int(R), ctypes.c_uint64(seed),
                                  ctypes.byref(rid)), "engine_submit")
    eng.requests[rid.value] = (pb, int(R), pb.n, bool(pb.info().is_integer))
    return rid.value


def engine_step(eng: Engine, stream=None, cap=4096):
    """Ids of the requests that finished in this step.  On TIMEOUT the raised
    SBQAError carries them as ``done_ids`` (failed ones included)."""
    n = ctypes.c_int32()
    ids = np.empty(cap, dtype=np.int32)
    st = lib.sbqa_engine_step(eng.handle, _stream(stream) or None, ctypes.byref(n), _p(ids, ctypes.c_int32),
                              int(cap))
    done = ids[:min(n.value, cap)].tolist()
    if st != OK:
        err = SBQAError(st, "engine_step", lib.sbqa_last_error().decode())
        err.done_ids = done
        raise err
    return done


def engine_result(eng: Engine, rid):
    if rid not in eng.requests:
        _check(lib.sbqa_engine_result(eng.handle, int(rid), None, None, None, None), "engine_result")
    _, R, N, _ = eng.requests[rid]
    spins = np.empty((R, N), dtype=np.int8)
    e = np.empty(R)
    ei = np.zeros(R, dtype=np.int64)
    k = np.empty(R, dtype=np.int32)
    _check(lib.sbqa_engine_result(eng.handle, int(rid), _p(spins, ctypes.c_int8), _p(e, ctypes.c_double),
                                  _p(ei, ctypes.c_int64), _p(k, ctypes.c_int32)), "engine_result")
    return {"spins": spins, "energy": e, "energy_int": ei, "replica": k}


def engine_stats(eng: Engine):
    st = EngineStats()
    _check(lib.sbqa_engine_stats(eng.handle, ctypes.byref(st)), "engine_stats")
    return {f: getattr(st, f) for f, _ in EngineStats._fields_}
