"""GB300 (sm_103a) implementation of the numeric phase of HYLU (X. Chen,
"HYLU: Hybrid Parallel Sparse LU Factorization"): up-looking sparse LU with
row-row / sup-row kernels and supernode diagonal pivoting (Sec. 2.2), its
forward/backward and transpose substitution with FP64 iterative refinement
(Sec. 2.3), behind the C ABI of include/hylu.h.

This package is a thin binding: ``capi`` marshals arguments to the C ABI of
libhylu.so (same function names); ``Solver`` wraps a handle for torch CUDA
tensors.  Every numeric step runs in the library's CUDA kernels; importing
the binding raises if the library cannot be loaded.
"""
from .capi import (HYLU_OK, HyluError, Info, Options, default_options, hylu_analyze, hylu_destroy,
                   hylu_export_factors, hylu_export_pattern, hylu_export_perm, hylu_factor,
                   hylu_get_info, hylu_grad_values, hylu_launch_count, hylu_measure_fp64_peak, hylu_refactor, hylu_solve, hylu_solve_transpose,
                   library_path, load)
from .solver import BatchSolver, Solver, analyze
from .autograd import HyluSolve, solve

__all__ = [
    "HYLU_OK", "HyluError", "Info", "Options", "default_options", "hylu_analyze", "hylu_destroy",
    "hylu_export_factors", "hylu_export_pattern", "hylu_export_perm", "hylu_factor", "hylu_get_info",
    "hylu_grad_values",
    "hylu_launch_count", "hylu_measure_fp64_peak", "hylu_refactor", "hylu_solve", "hylu_solve_transpose", "library_path", "load",
    "Solver", "BatchSolver", "analyze", "HyluSolve", "solve",
]
