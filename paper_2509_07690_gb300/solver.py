"""Handle wrapper for torch CUDA tensors (torch supplies device memory and
streams only; every numeric step runs in libhylu's kernels)."""
from __future__ import annotations

import numpy as np

from . import capi


def _stream(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


class Solver:
    """One analysed sparsity pattern (hylu_analyze) and its device factors."""

    def __init__(self, n, rowptr, col, vals=None, user_perm=None, **opts):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.opt = capi.default_options(**opts)
        self.h = capi.hylu_analyze(self.n, self.rowptr, self.col, vals, user_perm, self.opt)
        self.info = capi.hylu_get_info(self.h)
        self._factored = False

    # ------------------------------------------------------------ numeric
    def factor(self, d_vals, stream=None):
        """d_vals: torch float64 CUDA tensor of the nnz values (CSR order)."""
        assert d_vals.is_cuda and d_vals.dtype.itemsize == 8 and d_vals.is_contiguous()
        fn = capi.hylu_refactor if self._factored else capi.hylu_factor
        rc = fn(self.h, d_vals.data_ptr(), _stream(stream))
        self._factored = True
        return rc

    def solve(self, d_b, d_x=None, stream=None, transpose=False):
        """d_b: float64 CUDA tensor [n] or [nrhs, n] (each right-hand side
        contiguous).  Returns d_x of the same shape."""
        import torch
        b2 = d_b.reshape(-1, self.n)
        assert b2.is_contiguous()
        if d_x is None:
            d_x = torch.empty_like(d_b)
        x2 = d_x.reshape(-1, self.n)
        fn = capi.hylu_solve_transpose if transpose else capi.hylu_solve
        self.last_rc = fn(self.h, b2.data_ptr(), x2.data_ptr(), b2.shape[0], self.n, _stream(stream))
        return d_x

    def get_info(self) -> capi.Info:
        self.info = capi.hylu_get_info(self.h)
        return self.info

    # ------------------------------------------------------------ export
    def export_perm(self):
        return capi.hylu_export_perm(self.h, self.n, self.info.nnodes)

    def export_pattern(self):
        return capi.hylu_export_pattern(self.h, self.n, self.info.nnz_store)

    def export_factors(self):
        return capi.hylu_export_factors(self.h, self.n, self.info.nnz_store)

    def close(self):
        if getattr(self, "h", None):
            capi.hylu_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def analyze(n, rowptr, col, vals=None, user_perm=None, **opts) -> Solver:
    return Solver(n, rowptr, col, vals, user_perm, **opts)
