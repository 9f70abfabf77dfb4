"""GB300 (sm_103a) hot path of Simulated Bifurcation Quantum Annealing.

Simulated Bifurcation Quantum Annealing (arXiv 2604.01050): simulated
bifurcation with a ferromagnetic coupling between Trotter replicas along a
periodic imaginary-time axis.  The hot path -- initial state, the
time-stepped equations of motion (coupling product, replica coupling,
symplectic update, wall, threshold) and the readout (sign, Ising energies,
best per run) -- runs in the hand-written CUDA kernels of ``libsbqa.so``,
whose C ABI is declared in ``include/sbqa.h``.  This package is the thin
Python binding of that ABI; it has no CPU fallback.

``paper_2604_01050_gb300.build`` compiles the library and can be imported
before it exists; every other name loads ``libsbqa.so`` on first use and
raises ImportError if it has not been built.
"""
import importlib

_binding = None


def __getattr__(name):
    global _binding
    if name.startswith("__"):
        raise AttributeError(name)
    if name == "build":
        return importlib.import_module(".build", __name__)
    if _binding is None:
        _binding = importlib.import_module("._binding", __name__)
    try:
        return getattr(_binding, name)
    except AttributeError:
        raise AttributeError("module %r has no attribute %r" % (__name__, name)) from None
