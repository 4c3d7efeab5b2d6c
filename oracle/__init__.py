"""ORACLE -- test infrastructure only.

A plain, slow, FP64 CPU implementation of the non-recursive N-dimensional
Bartels-Stewart method (Cuesta & de la Hoz, arXiv 2412.15840).  Only the tests,
`__graft_entry__.smoke()` and the CPU-baseline / reference leg of `bench.py` may
import it.  The CUDA library shares no code with it and never calls it.

Pinned by the `-m "not gpu"` tests in tests/test_oracle.py against: the
worked index example of Section 2.2 (golden fixture), a dense solve of the
Kronecker-sum system of Eq. (systvec), the classical 2-D Sylvester solver
(Eq. (sylvester)), the FFT closed form for circulant operators and the
diagonal closed form (Remark 1), the singleton reduction, the residual
invariant, the nested-loop Algorithm 1, and planted mistakes.  The ODE solution of
Theorem 1 (`evolve`) is pinned against the exponential of the augmented
Kronecker-sum matrix, the scalar closed form for diagonal operators, a
fourth-order Runge-Kutta integration (the experiment of Section 5.2), its
t = 0 and steady-state limits, and planted mistakes.  The real-arithmetic
variant (`real_variant`: real Schur factors, quasi-triangular sweep) is pinned
in tests/test_oracle_real.py against the dense Kronecker-sum solve (of A_j and
of the T_j), the classical 2-D Sylvester solver, the complex oracle's solution
of the same real problem, orthogonality of the transforms, and planted
mistakes (block coupling dropped, factor transposed).
"""
from .bartels_stewart import (  # noqa: F401
    linear_index,
    counter_order,
    mode_product,
    apply_operator,
    residual,
    schur_factors,
    forward_transform,
    triangular_sweep,
    triangular_sweep_nested,
    back_transform,
    solve,
    solve_with_factors,
    evolve,
    evolve_rhs,
    rel_err,
    backward_error,
    set_threads,
)
