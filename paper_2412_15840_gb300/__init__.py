"""GB300 (sm_103a) solver for N-dimensional Sylvester tensor equations

    sum_j A_j (x)_j X = B

by the non-recursive Bartels-Stewart method (forward transform by the Schur
factors, triangular sweep, back transform), with a plain FP64 path and an
FP32 path refined to FP64 accuracy by FP64 residuals, and the solution at
any time t of the linear ODE X_t = sum_j A_j (x)_j X + B (Theorem 1).  The compute runs in
libsylv.so (C ABI in include/sylv.h); this package only marshals arguments.
"""
from .binding import (  # noqa: F401
    EXPORTED,
    PHASES,
    Plan,
    SylvError,
    expm,
    from_device,
    lib,
    schur,
    schur_real,
    solve_batched,
    to_device,
    workspace_size_batched,
)

__all__ = ["Plan", "SylvError", "schur", "schur_real", "expm", "solve_batched", "workspace_size_batched",
           "to_device", "from_device", "lib", "EXPORTED", "PHASES"]
