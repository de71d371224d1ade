"""GB300-native Lattice Boltzmann Relaxation Scheme (LBRS) for inviscid compressible flow.

The time step (streaming, boundary conditions, moments, Euler fluxes,
algebraic equilibria, relaxation) runs in hand-written CUDA kernels for
sm_103a behind the C ABI of include/lbrs.h (liblbrs.so, built in-tree by
``paper_1504_07034_gb300.build``).  ``abi`` is the ctypes binding with the C
names; ``Solver`` wraps it with torch tensors.
"""
import importlib

__all__ = ["Solver", "abi", "build"]


def __getattr__(name):
    if name == "Solver":
        return importlib.import_module(".solver", __name__).Solver
    if name in ("abi", "solver"):
        return importlib.import_module("." + name, __name__)
    if name == "build":
        return importlib.import_module(".build", __name__).build
    raise AttributeError(name)
