"""Reader of the analysis image that hylu_plan_save writes, for host tests of
the plan's schedules.  The field order is the library serializer's (options,
plan scalars, plan arrays, batch layout); the reader checks that it consumed
every byte before the checksum, so a change of layout fails loudly here."""
from __future__ import annotations

import struct

import numpy as np

_OPTS = [("ordering", "i"), ("static_pivot", "i"), ("scale", "i"), ("sn_max", "i"), ("nd_leaf", "i"),
         ("pivot_tau", "d"), ("refine_tol", "d"), ("refine_maxit", "i"), ("refine", "i"),
         ("spin_limit", "q"), ("rows_per_task", "i"), ("debug", "i"), ("amd_dense", "d"), ("timing", "i"),
         ("precision", "i"), ("heavy_ratio", "d"), ("gemm_min_rows", "i"), ("solve_seq_rows", "i")]
_SCALARS = [("n", "i"), ("nnz_a", "q"), ("nnodes", "i"), ("nnz_l", "q"), ("nnz_panel", "q"),
            ("nnz_store", "q"), ("nnz_f", "q"), ("flops_unpadded", "d"), ("flops_padded", "d"),
            ("n_tasks", "i"), ("row_levels", "i"), ("flops_row_row", "d"), ("flops_sup_row", "d"),
            ("flops_sup_sup", "d"), ("flops_in_sn", "d"), ("ordering", "i"), ("max_row", "i"), ("max_sn", "i"),
            ("analyze_ms", "d"), ("analyze_phase_ms", "4d")]
I32, I64, F64 = np.int32, np.int64, np.float64
_ARRAYS = [("a_rp", I64), ("a_ci", I32), ("rowperm", I32), ("colperm", I32), ("dr", F64), ("dc", F64),
           ("ah_rp", I64), ("ah_slot", I32), ("ah_src", I64), ("ah_scale", F64),
           ("sn_start", I32), ("node_of", I32), ("row_lptr", I64), ("lcols", I32), ("node_tail_off", I64),
           ("tcols", I32), ("node_panel_off", I64), ("row_flops", F64),
           ("node_ntask", I32), ("task_node", I32), ("task_chunk", I32), ("task_level", I32),
           ("row_order", I32), ("heavy_order", I32), ("heavy_rank", I32), ("row_level", I32),
           ("fwd_order", I32), ("bwd_order", I32), ("fwd_level", I32), ("bwd_level", I32),
           ("fwd_count", I32), ("bwd_count", I32), ("ut_order", I32), ("lt_order", I32),
           ("ut_level", I32), ("lt_level", I32), ("ut_count", I32), ("lt_count", I32),
           ("node_inst", I32), ("fwd_off", I32), ("bwd_off", I32), ("ut_off", I32), ("lt_off", I32)]
_BATCH = [("batch", "i"), ("k", "i"), ("nsets", "i"), ("pos_n", "i")]
_BATCH_ARRAYS = [("row_base", I32), ("node_base", I32), ("val_base", I64)]


class PlanImage:
    """Every field of an image as an attribute (options under .opt)."""

    def __init__(self, image: bytes):
        assert image[:8] == b"HYLUPLAN"
        self._b = image
        self._p = 8
        version, order = self._scalar("I"), self._scalar("I")
        assert version == 3 and order == 0x01020304
        self.opt = {name: self._scalar(f) for name, f in _OPTS}
        for name, f in _SCALARS:
            setattr(self, name, self._scalar(f))
        for name, dt in _ARRAYS:
            setattr(self, name, self._array(dt))
        for name, f in _BATCH:
            setattr(self, name, self._scalar(f))
        for name, dt in _BATCH_ARRAYS:
            setattr(self, name, self._array(dt))
        assert self._p == len(image) - 8, "image layout differs from the reader's"

    def _scalar(self, f):
        size = struct.calcsize("<" + f)
        v = struct.unpack_from("<" + f, self._b, self._p)
        self._p += size
        return v[0] if len(v) == 1 else v

    def _array(self, dt):
        (count,) = struct.unpack_from("<Q", self._b, self._p)
        self._p += 8
        nbytes = count * np.dtype(dt).itemsize
        a = np.frombuffer(self._b, dtype=dt, count=count, offset=self._p).copy()
        self._p += nbytes
        return a

    # instance of every node and each instance's slice of a per-level count array
    def node_instance(self) -> np.ndarray:
        return self.node_inst if len(self.node_inst) else np.zeros(self.nnodes, np.int32)

    def slices(self, kind: str) -> np.ndarray:
        off = getattr(self, kind + "_off")
        count = getattr(self, kind + "_count")
        return off if len(off) else np.array([0, len(count)], np.int32)
