"""GB300-native tensor-product B-spline smoothing with a matrix-free multigrid-preconditioned CG.

The solver lives in the CUDA library libsps.so (C ABI in include/sps.h);
`binding` is its thin ctypes front end.  Build the library with
`paper_1901_00654_gb300.build.build_library()`.
"""
__all__ = ["binding", "build"]
