"""Handle wrapper for torch CUDA tensors (torch supplies device memory and
streams only; every numeric step runs in libhylu's kernels)."""
from __future__ import annotations

import numpy as np

from . import capi


def _stream(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _device_f64(t, what: str, numel: int | None = None, multiple_of: int | None = None):
    """The kernels read and write exactly the sizes the handle implies, so
    a tensor of another type, layout or size is refused here."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{what}: expected a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what}: expected {numel} values, got {t.numel()}")
    if multiple_of == 0 and t.numel() != 0:
        raise ValueError(f"{what}: an empty system takes empty tensors, got {t.numel()} values")
    if multiple_of and (t.numel() == 0 or t.numel() % multiple_of):
        raise ValueError(f"{what}: expected a positive multiple of {multiple_of} values, got {t.numel()}")


def _nrhs(t, n: int) -> int:
    """Right-hand sides in a [n] or [nrhs, n] tensor (n = 0: from its shape)."""
    if n:
        return t.numel() // n
    return t.shape[0] if t.dim() == 2 else 1


class Solver:
    """One analysed sparsity pattern (hylu_analyze) and its device factors."""

    def __init__(self, n, rowptr, col, vals=None, user_perm=None, **opts):
        self.n = int(n)
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.nnz = int(self.rowptr[-1])
        self.opt = capi.default_options(**opts)
        self.h = capi.hylu_analyze(self.n, self.rowptr, self.col, vals, user_perm, self.opt)
        self.info = capi.hylu_get_info(self.h)
        self._factored = False
        self.factor_gen = 0      # factorizations issued on this handle

    @classmethod
    def from_csr(cls, A, **opts) -> "Solver":
        """A solver for a square CSR matrix given as any object with
        indptr / indices / data (scipy.sparse.csr_matrix, for one).  Column
        indices are sorted per row on a copy (the analysis requires them
        sorted); duplicate entries are refused by the analysis.  The values
        in that sorted order are kept as `values`: factor() takes them (or
        later value sets in the same order) as a CUDA tensor."""
        n = int(A.shape[0])
        if A.shape[0] != A.shape[1]:
            raise ValueError(f"from_csr: the matrix must be square, got {A.shape}")
        rowptr = np.asarray(A.indptr, dtype=np.int64)
        col = np.asarray(A.indices, dtype=np.int32).copy()
        val = np.asarray(A.data, dtype=np.float64).copy()
        for i in range(n):
            a, b = rowptr[i], rowptr[i + 1]
            if b - a > 1 and np.any(np.diff(col[a:b]) < 0):
                o = np.argsort(col[a:b], kind="stable")
                col[a:b] = col[a:b][o]
                val[a:b] = val[a:b][o]
        s = cls(n, rowptr, col, val, **opts)
        s.values = val
        return s

    # ------------------------------------------------------------ checkpoint
    def save(self, path=None) -> bytes:
        """The analysis as a byte image (hylu_plan_save), also written to
        `path` when one is given."""
        image = capi.hylu_plan_save(self.h)
        if path is not None:
            with open(path, "wb") as f:
                f.write(image)
        return image

    @classmethod
    def load(cls, source, **opts) -> "Solver":
        """A solver from a saved analysis (hylu_plan_load): `source` is the
        byte image or a path to it.  Keyword options set the numeric options
        (as for the constructor); without any, the saved options are kept.
        An image of a batch gives a solver over the combined system."""
        if isinstance(source, (bytes, bytearray, memoryview)):
            image = bytes(source)
        else:
            with open(source, "rb") as f:
                image = f.read()
        self = cls.__new__(cls)
        self.opt = capi.default_options(**opts) if opts else None
        self.h = capi.hylu_plan_load(image, self.opt)
        self.info = capi.hylu_get_info(self.h)
        self.n = int(self.info.n)
        self.nnz = int(self.info.nnz_a)
        self.rowptr = None
        self.col = None
        self._factored = False
        self.factor_gen = 0
        return self

    # ------------------------------------------------------------ numeric
    def factor(self, d_vals, stream=None):
        """d_vals: torch float64 CUDA tensor of the nnz values (CSR order)."""
        _device_f64(d_vals, "d_vals", numel=self.nnz)
        fn = capi.hylu_refactor if self._factored else capi.hylu_factor
        rc = fn(self.h, d_vals.data_ptr(), _stream(stream))
        self._factored = True
        self.factor_gen += 1
        return rc

    def solve(self, d_b, d_x=None, stream=None, transpose=False):
        """d_b: float64 CUDA tensor [n] or [nrhs, n] (each right-hand side
        contiguous).  Returns d_x of the same shape."""
        import torch
        _device_f64(d_b, "d_b", multiple_of=self.n)
        if d_x is None:
            d_x = torch.empty_like(d_b)
        _device_f64(d_x, "d_x", numel=d_b.numel())
        nbytes = 8 * d_b.numel()
        if nbytes and d_x.data_ptr() < d_b.data_ptr() + nbytes and d_b.data_ptr() < d_x.data_ptr() + nbytes:
            raise ValueError("solve: d_b and d_x overlap (the solution may not be written over the right-hand side)")
        fn = capi.hylu_solve_transpose if transpose else capi.hylu_solve
        self.last_rc = fn(self.h, d_b.data_ptr(), d_x.data_ptr(), _nrhs(d_b, self.n), self.n, _stream(stream))
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


class BatchSolver(Solver):
    """k systems x nsets value sets in one block-diagonal plan
    (hylu_analyze_batch): one persistent launch factors every instance;
    instance q = v * k + s occupies rows row_base[q] .. of the combined
    system and values val_base[q] .. of the concatenated value array."""

    def __init__(self, systems, nsets: int = 1, **opts):
        self.opt = capi.default_options(**opts)
        self.systems = systems
        self.k = len(systems)
        self.nsets = int(nsets)
        self.h = capi.hylu_analyze_batch(systems, self.nsets, self.opt)
        self.info = capi.hylu_get_info(self.h)
        self.row_base, self.val_base, self.n = capi.hylu_batch_layout(self.h, self.k * self.nsets)
        rps = []
        off = 0
        for v in range(self.nsets):
            for (n, rp, ci, _) in systems:
                rps.append(np.asarray(rp, np.int64)[1:] + off)
                off += int(rp[-1])
        self.rowptr = np.concatenate([[0]] + rps).astype(np.int64)
        self.nnz = int(self.rowptr[-1])
        self.col = None
        self._factored = False
        self.factor_gen = 0

    @classmethod
    def load(cls, source, **opts):
        raise TypeError("BatchSolver.load: load a batch image with Solver.load (a solver over the combined system)")

    def concat_values(self, value_sets):
        """value_sets[v][s]: values of system s in value set v -> one array."""
        return np.concatenate([np.asarray(value_sets[v][s], np.float64)
                               for v in range(self.nsets) for s in range(self.k)])

    def tune(self, d_vals, stream=None) -> int:
        _device_f64(d_vals, "d_vals", numel=self.nnz)
        self._factored = True
        self.factor_gen += 1
        return capi.hylu_tune(self.h, d_vals.data_ptr(), _stream(stream))

    def graph_capture(self, d_vals, d_b, d_x, corrections: int = 0, stream=None):
        """Record refactor + solve (+ `corrections` fixed FP64 refinement
        steps, then the residual norms get_info reports) as a CUDA graph."""
        _device_f64(d_vals, "d_vals", numel=self.nnz)
        _device_f64(d_b, "d_b", multiple_of=self.n)
        _device_f64(d_x, "d_x", numel=d_b.numel())
        capi.hylu_graph_capture(self.h, d_vals.data_ptr(), d_b.data_ptr(), d_x.data_ptr(), _nrhs(d_b, self.n),
                                self.n, int(corrections), _stream(stream))

    def graph_launch(self, stream=None):
        capi.hylu_graph_launch(self.h, _stream(stream))
