"""Plain FP64 CPU oracle of the SBQA hot path (test infrastructure only).

This package is the independent restatement of Simulated Bifurcation Quantum
Annealing (arXiv 2604.01050, Sec. II A-B) that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU baseline leg
of ``bench.py`` may import it; the product library never does.  It shares no
code with ``paper_2604_01050_gb300``: the arithmetic lives in
``sbqa_oracle.c`` (plain C, FP64, no FMA contraction) and this module only
builds it and marshals numpy arrays.

Functions and the passages they follow:
  splitmix64, init_state   random initial state (Sec. II A), SplitMix64
                           (Steele, Lea & Flood 2014) as counter-based source
  schedule, jperp, gamma   a(t)=t/T, Gamma_x(t), J_perp(t) (Eq. 5, Eq. S12),
                           Delta(t) = 0.7 t/T (after Eq. 8)
  f                        thresholded f (Eq. 8) / bSB f(x)=x (after Eq. 3)
  force, step, run         SBQA equations of motion (Eqs. 6-7), symplectic
                           Euler, wall rule (after Eq. 3)
  energy, energy_int       Ising energy with the Eq. 4 / Eq. S1 sign
  brute_force              exhaustive ground state (small N)
  gap, tte                 optimality gap (Eq. 9), time-to-epsilon (Eq. 10)
  round_bf16               RNE rounding to bfloat16 (quantisation of J for the
                           BF16 product)

Every function has a pin in ``tests/test_oracle_pins.py`` against something
other than itself (published vectors, closed forms, symmetries, the plain-SB
reduction, the Hamiltonian gradient, brute force).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbqa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_i64_p = ctypes.POINTER(ctypes.c_int64)
_c_i32_p = ctypes.POINTER(ctypes.c_int32)
_c_i8_p = ctypes.POINTER(ctypes.c_int8)


def build(force: bool = False) -> str:
    """Compile sbqa_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("row_ptr", _c_i64_p), ("col", _c_i32_p),
                ("val", _c_double_p), ("h", _c_double_p)]


class _Params(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("c0", ctypes.c_double),
                ("dt", ctypes.c_double), ("variant", ctypes.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_splitmix64.restype = ctypes.c_uint64
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_uniform_f32.restype = ctypes.c_float
        lib.orc_uniform_f32.argtypes = [ctypes.c_uint64, ctypes.c_float]
        lib.orc_init_state.restype = None
        lib.orc_init_state.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, _c_double_p, _c_double_p]
        lib.orc_round_bf16.restype = ctypes.c_double
        lib.orc_round_bf16.argtypes = [ctypes.c_double]
        lib.orc_jperp.restype = ctypes.c_double
        lib.orc_jperp.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.orc_gamma.restype = ctypes.c_double
        lib.orc_gamma.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
        lib.orc_schedule.restype = None
        lib.orc_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, _c_double_p, _c_double_p, ctypes.c_int,
                                     _c_double_p, _c_double_p, _c_double_p]
        lib.orc_c0_auto.restype = ctypes.c_double
        lib.orc_c0_auto.argtypes = [ctypes.POINTER(_Problem)]
        lib.orc_f.restype = ctypes.c_double
        lib.orc_f.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.orc_force.restype = None
        lib.orc_force.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Params), ctypes.c_int,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  _c_double_p, _c_double_p]
        lib.orc_step_run.restype = None
        lib.orc_step_run.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Params), ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     _c_double_p, _c_double_p]
        lib.orc_energy.restype = ctypes.c_double
        lib.orc_energy.argtypes = [ctypes.POINTER(_Problem), _c_i8_p]
        lib.orc_energy_int.restype = ctypes.c_int64
        lib.orc_energy_int.argtypes = [ctypes.POINTER(_Problem), _c_i8_p]
        lib.orc_brute_force.restype = ctypes.c_double
        lib.orc_brute_force.argtypes = [ctypes.POINTER(_Problem), _c_i8_p]
        lib.orc_run.restype = None
        lib.orc_run.argtypes = [
            ctypes.POINTER(_Problem), ctypes.POINTER(_Params), ctypes.c_int, ctypes.c_int,
            ctypes.c_int, _c_double_p, _c_double_p, ctypes.c_double, ctypes.c_double,
            ctypes.c_int, ctypes.c_int, ctypes.c_int, _c_double_p, _c_double_p, ctypes.c_int,
            _c_double_p, _c_double_p, ctypes.c_int, ctypes.c_int, _c_double_p, _c_i64_p,
            _c_double_p, _c_i32_p, _c_i32_p, _c_i8_p]
        _lib = lib
        return lib


def _ptr(a, ctype):
    if a is None:
        return ctypes.cast(None, ctypes.POINTER(ctype))
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Problem:
    """Ising instance (J symmetric, zero diagonal, h) held as CSR in FP64."""

    def __init__(self, n, row_ptr, col, val, h=None):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
        self.is_integer = bool(np.all(self.val == np.round(self.val)) and
                               (self.h is None or np.all(self.h == np.round(self.h))))
        self._c = _Problem(self.n, _ptr(self.row_ptr, ctypes.c_int64), _ptr(self.col, ctypes.c_int32),
                           _ptr(self.val, ctypes.c_double), _ptr(self.h, ctypes.c_double))

    @classmethod
    def dense(cls, J, h=None):
        J = np.asarray(J, dtype=np.float64)
        n = J.shape[0]
        rows, cols = np.nonzero(J)
        row_ptr = np.zeros(n + 1, dtype=np.int64)
        np.add.at(row_ptr, rows + 1, 1)
        return cls(n, np.cumsum(row_ptr), cols, J[rows, cols], h)

    @classmethod
    def csr(cls, n, row_ptr, col, val, h=None):
        return cls(n, row_ptr, col, val, h)

    def to_dense(self):
        J = np.zeros((self.n, self.n))
        for i in range(self.n):
            a, b = self.row_ptr[i], self.row_ptr[i + 1]
            J[i, self.col[a:b]] = self.val[a:b]
        return J

    def bf16(self):
        """The same instance with J rounded to bfloat16 (h unchanged)."""
        return Problem(self.n, self.row_ptr, self.col, round_bf16(self.val), self.h)


def splitmix64(seed: int, ctr: int) -> int:
    return int(_load().orc_splitmix64(ctypes.c_uint64(seed), ctypes.c_uint64(ctr)))


def uniform_f32(z: int, amp: float) -> float:
    return float(_load().orc_uniform_f32(ctypes.c_uint64(z), ctypes.c_float(amp)))


def init_state(seed, N, P, R, amp=0.1):
    """Initial (x, y), each shaped (R, P, N), FP32 values widened to FP64."""
    x = np.empty((R, P, N)); y = np.empty((R, P, N))
    _load().orc_init_state(ctypes.c_uint64(seed), N, P, R, amp,
                           _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double))
    return x, y


def round_bf16(v):
    lib = _load()
    v = np.asarray(v, dtype=np.float64)
    return np.vectorize(lambda t: lib.orc_round_bf16(float(t)), otypes=[np.float64])(v) if v.size else v.copy()


def jperp(beta, gamma, P):
    return _load().orc_jperp(beta, gamma, P)


def gamma(gamma0, alpha, tau):
    return _load().orc_gamma(gamma0, alpha, tau)


def f(x, delta, variant=0):
    return _load().orc_f(float(x), float(delta), int(variant))


def schedule(S, P, R, beta, alpha, gamma0=1.0, delta_slope=0.7, jperp_enable=True):
    """(a[S], delta[S+1], jperp[R, S]) in FP64."""
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    a = np.empty(S); d = np.empty(S + 1); jp = np.empty((R, S))
    _load().orc_schedule(S, P, R, gamma0, delta_slope, _ptr(beta, ctypes.c_double),
                         _ptr(alpha, ctypes.c_double), int(bool(jperp_enable)),
                         _ptr(a, ctypes.c_double), _ptr(d, ctypes.c_double), _ptr(jp, ctypes.c_double))
    return a, d, jp


def c0_auto(pb: Problem) -> float:
    return _load().orc_c0_auto(ctypes.byref(pb._c))


def _params(a0, c0, dt, variant):
    return _Params(a0, c0, dt, variant)


def force(pb: Problem, x, P, a_n, delta_n, jp, a0=1.0, c0=None, dt=0.5, variant=0):
    """Right-hand side of Eq. 7 for one run; x shaped (P, N)."""
    c0 = c0_auto(pb) if c0 is None else c0
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    pp = _params(a0, c0, dt, variant)
    _load().orc_force(ctypes.byref(pb._c), ctypes.byref(pp), P, a_n, delta_n, jp,
                      _ptr(x, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def step(pb: Problem, x, y, P, a_n, delta_n, jp, a0=1.0, c0=None, dt=0.5, variant=0):
    """One symplectic-Euler step + wall of one run, returns new (x, y)."""
    c0 = c0_auto(pb) if c0 is None else c0
    x = np.array(x, dtype=np.float64, order="C"); y = np.array(y, dtype=np.float64, order="C")
    pp = _params(a0, c0, dt, variant)
    _load().orc_step_run(ctypes.byref(pb._c), ctypes.byref(pp), P, a_n, delta_n, jp,
                         _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double))
    return x, y


def energy(pb: Problem, s) -> float:
    s = np.ascontiguousarray(s, dtype=np.int8)
    return _load().orc_energy(ctypes.byref(pb._c), _ptr(s, ctypes.c_int8))


def energy_int(pb: Problem, s) -> int:
    s = np.ascontiguousarray(s, dtype=np.int8)
    return int(_load().orc_energy_int(ctypes.byref(pb._c), _ptr(s, ctypes.c_int8)))


def energies(pb: Problem, spins):
    """Energies of many spin vectors, spins shaped (..., N)."""
    spins = np.asarray(spins, dtype=np.int8)
    flat = spins.reshape(-1, pb.n)
    fn = energy_int if pb.is_integer else energy
    out = np.array([fn(pb, s) for s in flat], dtype=np.int64 if pb.is_integer else np.float64)
    return out.reshape(spins.shape[:-1])


def brute_force(pb: Problem):
    """(ground energy, one ground state) by enumeration; N <= 30."""
    if pb.n > 30:
        raise ValueError("brute force limited to N <= 30")
    s = np.empty(pb.n, dtype=np.int8)
    e = _load().orc_brute_force(ctypes.byref(pb._c), _ptr(s, ctypes.c_int8))
    return e, s


def run(pb: Problem, S, P, R, seed, beta, alpha, a0=1.0, c0=None, dt=0.5, gamma0=1.0,
        delta_slope=0.7, amp=0.1, jperp_enable=True, variant=0, n_begin=0, n_end=None,
        x0=None, y0=None, n_traj=0, eval_every=0, best=None):
    """Run steps [n_begin, n_end) of an S-step anneal of R runs x P replicas.

    x0, y0 (R, P, N) default to the seeded initial state.  Returns a dict with
    the final x, y, the trajectory of the first n_traj steps, the R*P final
    energies and the per-run best (energy, replica k, step, spins).
    ``best`` (a previous result dict) carries the best-so-far into a resumed
    range.
    """
    lib = _load()
    n_end = S if n_end is None else n_end
    c0 = c0_auto(pb) if c0 is None else c0
    N = pb.n
    if x0 is None:
        x, y = init_state(seed, N, P, R, amp)
    else:
        x = np.array(x0, dtype=np.float64, order="C").reshape(R, P, N)
        y = np.array(y0, dtype=np.float64, order="C").reshape(R, P, N)
    beta = np.ascontiguousarray(np.broadcast_to(np.asarray(beta, dtype=np.float64), (R,)))
    alpha = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, dtype=np.float64), (R,)))
    nt = max(0, min(int(n_traj), n_end - n_begin))
    tx = np.empty((nt, R, P, N)) if nt else None
    ty = np.empty((nt, R, P, N)) if nt else None
    e = np.empty((R, P)); ei = np.zeros((R, P), dtype=np.int64)
    if best is None:
        be = np.full(R, np.inf); bk = np.full(R, -1, dtype=np.int32)
        bs_ = np.full(R, -2, dtype=np.int32); bsp = np.zeros((R, N), dtype=np.int8)
    else:
        be = best["best_energy"].copy(); bk = best["best_k"].copy()
        bs_ = best["best_step"].copy(); bsp = best["best_spins"].copy()
    pp = _params(a0, c0, dt, variant)
    lib.orc_run(ctypes.byref(pb._c), ctypes.byref(pp), S, P, R, _ptr(beta, ctypes.c_double),
                _ptr(alpha, ctypes.c_double), gamma0, delta_slope, int(bool(jperp_enable)),
                n_begin, n_end, _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double), nt,
                _ptr(tx, ctypes.c_double), _ptr(ty, ctypes.c_double), int(eval_every),
                int(pb.is_integer), _ptr(e, ctypes.c_double), _ptr(ei, ctypes.c_int64),
                _ptr(be, ctypes.c_double), _ptr(bk, ctypes.c_int32), _ptr(bs_, ctypes.c_int32),
                _ptr(bsp, ctypes.c_int8))
    return {"x": x, "y": y, "traj_x": tx, "traj_y": ty, "energy": e,
            "energy_int": ei if pb.is_integer else None, "best_energy": be, "best_k": bk,
            "best_step": bs_, "best_spins": bsp, "c0": c0}


def gap(E, E0):
    """Optimality gap g = (E - E0) / |E0|  (Eq. 9)."""
    return (E - E0) / abs(E0)


def tte(tau, p_success, p_target=0.99):
    """Time-to-epsilon (Eq. 10): tau * log(1 - p_target) / log(1 - p_success).

    Readings: p_success == 0 gives +inf; p_success >= p_target gives tau (one
    run already reaches the target probability)."""
    if p_success <= 0.0:
        return math.inf
    if p_success >= p_target:
        return float(tau)
    return tau * math.log(1.0 - p_target) / math.log(1.0 - p_success)
