"""GB300 (sm_103a) FP64 implementation of the hybrid DF + WENO-AO high-order finite-volume
scheme with GKS / L-F fluxes and S2O4 time stepping (arXiv 2402.10914).

The compute path is the CUDA library ``libdfgks.so`` behind the C ABI of ``include/dfgks.h``;
``solver.Solver`` is its thin Python front end.  ``inputs`` holds the seeded workloads.
Submodules are imported lazily so that ``inputs`` can be used without CUDA.
"""
__all__ = ["inputs", "solver", "build"]


def __getattr__(name):
    import importlib
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
