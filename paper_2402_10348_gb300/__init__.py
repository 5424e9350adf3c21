"""GB300-native (sm_103a) matrix-free Q1 residuals, Jacobian-vector products and
solvers of the fully Eulerian phase-field FSI method of Mao & Jaiman (arXiv 2402.10348).

The compute lives in libfsi.so (include/fsi.h); `paper_2402_10348_gb300.fsi` is its
Python binding.  Build the library with `paper_2402_10348_gb300._build.build()`.
"""
from . import fsi  # noqa: F401
