"""GB300-native DDM-GMRES solver for the Nedelec-discretised time-harmonic
Maxwell system (Beuchler, Kinnewig, Wick: optimized-Schwarz DDM with impedance
transmission, GMRES on the interface system, block-preconditioned GMRES in
every subdomain).

This package is a thin ctypes binding over the C ABI in include/thm.h
(libthm.so, built in-tree by `paper_2105_11993_gb300.build`).  Every step of
the solve runs in the library's CUDA kernels; PyTorch only provides device
memory and streams.  There is no CPU fallback: if the library is missing or no
GPU is present, the calls raise.
"""
from __future__ import annotations

from ._binding import (  # noqa: F401
    K_DDM, K_DOTS, K_KRYLOV, K_NAMES, K_PINV, K_SETUP, K_SPMV, K_UPDATE, LIB_PATH, MODE_FP64,
    MODE_MIXED, OP_KLOC, OP_PINV, OP_T, OP_TINV, PRECOND_BLOCKDIAG, PRECOND_FULL, TAG_DIRICHLET,
    TAG_IMPEDANCE, TAG_NATURAL, AssembleOptions, Mesh, SolveOptions, System, ThmError, algorithmic_bytes,
    factor_bytes, kernel_launches, load, profile_enable, profile_read, symbols, work_bytes,
)
