"""GB300-native walk-on-ellipsoids operator build, FP64 Jacobi SVD and TSVD
reconstruction for Cauchy-type inverse problems (arXiv:2409.03686).

``wos`` is the thin binding of the CUDA library (include/wos.h);
``workloads`` describes the seeded synthetic inputs.  Importing the package
loads nothing; the library is loaded on first use and raises if missing.
"""
__all__ = ["wos", "workloads", "build"]
