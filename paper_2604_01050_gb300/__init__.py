"""GB300 (sm_103a) hot path of Simulated Bifurcation Quantum Annealing.

Simulated Bifurcation Quantum Annealing (arXiv 2604.01050): simulated
bifurcation with a ferromagnetic coupling between Trotter replicas along a
periodic imaginary-time axis.  The hot path -- initial state, the
time-stepped equations of motion (coupling product, replica coupling,
symplectic update, wall, threshold) and the readout (sign, Ising energies,
best per run) -- runs in the hand-written CUDA kernels of ``libsbqa.so``,
whose C ABI is declared in ``include/sbqa.h``.  This package is the thin
Python binding of that ABI; it has no CPU fallback.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import (EXPORTS, LIB_PATH, Problem, SBQAError, create_problem_csr,  # noqa: F401
                       create_problem_dense, get_best, get_energies, get_state, run, run_advance,
                       run_begin, run_finish, set_schedule, set_state, synchronize, version)
