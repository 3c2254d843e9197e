"""GB300-native geometric multigrid for Q1 and rotated-Q1 finite element systems.

The solver is a C-ABI shared library (``include/mg.h``) of hand-written sm_103a CUDA
kernels; this package is a thin ctypes binding over it plus seeded input generators
(``workloads``). Importing the package loads nothing: the library is opened on first
use and an ImportError is raised if it has not been built.
"""
__all__ = ["workloads"]
