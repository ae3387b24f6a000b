"""GB300 (sm_103a) library for the k-th eigenvalue of symmetric kernel matrices
compressed as H^2-matrices: slicing the spectrum with the generalized
H^2-LDL^T factorization (Apriansyah & Yokota, arXiv 2311.08618).

The compute lives in ``libh2eig.so`` (CUDA kernels behind the C ABI of
``include/h2eig.h``); this package is a thin ctypes binding with the same
names.  There is no CPU fallback: loading fails loudly without the library.
"""
from .binding import (  # noqa: F401
    H2Error, H2Group, H2Matrix, Kernel, Options, lib, library_path,
    H2_K_LAPLACE_EPS, H2_K_YUKAWA_EPS, H2_K_GAUSS_PLUS_INV, H2_K_TRIDIAG_TEST, H2_K_MIN_TEST,
    H2_ADM_BOX, H2_ADM_CENTER, H2_ADM_WEAK, H2_PREC_FP64, H2_PREC_MIXED, H2_PREC_FP64_TC, EXPORTED_SYMBOLS,
)
