"""ctypes binding of include/hylu.h: one Python function per C entry point,
same names, argument marshalling only (host arrays as numpy, device arrays
and streams as integer addresses)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libhylu.so")
_lib = None

# the #define constants of include/hylu.h (a host test keeps the two in step)
HYLU_OK = 0
HYLU_WARN_PERTURBED = 1
HYLU_WARN_REFINE_STALLED = 2
HYLU_ERR_ARG = -1
HYLU_ERR_PATTERN = -2
HYLU_ERR_STRUCT_SINGULAR = -3
HYLU_ERR_NOMEM = -4
HYLU_ERR_CUDA = -5
HYLU_ERR_DEVICE_TIMEOUT = -6
HYLU_ERR_STATE = -7
HYLU_ERR_INTERNAL = -8
HYLU_ERR_TOO_LARGE = -9
HYLU_ORDER_AMD = 0
HYLU_ORDER_ND = 1
HYLU_ORDER_NATURAL = 2
HYLU_ORDER_USER = 3
HYLU_ORDER_AUTO = 4
HYLU_STATIC_SOLVE_MAX_N = 262144
ERRORS = {v: k for k, v in list(globals().items()) if k.startswith("HYLU_ERR_")}


class HyluError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("ordering", C.c_int), ("static_pivot", C.c_int), ("scale", C.c_int),
                ("sn_max", C.c_int), ("nd_leaf", C.c_int), ("pivot_tau", C.c_double),
                ("refine_tol", C.c_double), ("refine_maxit", C.c_int), ("refine", C.c_int),
                ("spin_limit", C.c_longlong), ("rows_per_task", C.c_int), ("debug", C.c_int),
                ("amd_dense", C.c_double), ("timing", C.c_int), ("precision", C.c_int),
                ("heavy_ratio", C.c_double), ("gemm_min_rows", C.c_int),
                ("solve_seq_rows", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz_a", C.c_int64), ("nnz_lu", C.c_int64),
                ("nnz_store", C.c_int64), ("nnodes", C.c_int32), ("nsupernodes", C.c_int32),
                ("rows_in_supernodes", C.c_int32), ("max_supernode", C.c_int32),
                ("ntasks", C.c_int32), ("flops", C.c_double), ("flops_padded", C.c_double),
                ("nperturb", C.c_int32), ("refine_iters", C.c_int32),
                ("backward_error", C.c_double), ("device_status", C.c_int32),
                ("failed_node", C.c_int32), ("analyze_ms", C.c_double),
                ("factor_kernel_ms", C.c_double), ("solve_kernel_ms", C.c_double),
                ("nheavy", C.c_int32), ("factor_levels", C.c_int32), ("fwd_levels", C.c_int32),
                ("bwd_levels", C.c_int32), ("flops_row_row", C.c_double), ("flops_sup_row", C.c_double),
                ("flops_sup_sup", C.c_double), ("flops_in_supernode", C.c_double), ("ordering", C.c_int32),
                ("analyze_phase_ms", C.c_double * 4), ("gemm_destinations", C.c_int32),
                ("gemm_tasks", C.c_int32), ("gemm_flops", C.c_double), ("tuned", C.c_int32),
                ("factor_blocks_per_sm", C.c_int32), ("solve_blocks_per_sm", C.c_int32),
                ("heavy_queue", C.c_int32), ("solve_seq_rows", C.c_int32),
                ("solve_segments", C.c_int32 * 2)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def library_path() -> str:
    return _SO


def load():
    """Load libhylu.so (built by paper_2509_07690_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_SO):
        raise ImportError(f"{_SO} is missing: run paper_2509_07690_gb300.build.build() first")
    lib = C.CDLL(_SO)
    H = C.c_void_p
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
    lib.hylu_default_options.argtypes = [C.POINTER(Options)]
    lib.hylu_analyze.argtypes = [C.c_int32, C.c_int64, i64p, i32p, C.c_void_p, C.c_void_p,
                                 C.POINTER(Options), C.POINTER(H)]
    lib.hylu_factor.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.hylu_refactor.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.hylu_solve.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    lib.hylu_solve_transpose.argtypes = [H, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    lib.hylu_get_info.argtypes = [H, C.POINTER(Info)]
    lib.hylu_export_perm.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hylu_export_pattern.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.hylu_export_schedule.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hylu_export_factors.argtypes = [H, C.c_void_p, C.c_void_p]
    lib.hylu_destroy.argtypes = [H]
    lib.hylu_launch_count.restype = C.c_int64
    lib.hylu_launch_count.argtypes = []
    lib.hylu_measure_fp64_peak.argtypes = [C.POINTER(C.c_double), C.c_void_p]
    lib.hylu_debug_gemm.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.POINTER(C.c_int32)]
    lib.hylu_export_gemm_plan.argtypes = [H, C.c_int, C.c_void_p, C.POINTER(C.c_int64)]
    lib.hylu_export_solve_segments.argtypes = [H, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_int64)]
    lib.hylu_split_gemm.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_int, C.c_void_p]
    lib.hylu_solve_static.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hylu_debug_trace.argtypes = [H, C.c_void_p]
    lib.hylu_grad_values.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]
    lib.hylu_analyze_batch.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                       C.POINTER(Options), C.POINTER(H)]
    lib.hylu_batch_layout.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.hylu_graph_capture.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                       C.c_void_p]
    lib.hylu_graph_launch.argtypes = [H, C.c_void_p]
    lib.hylu_tune.argtypes = [H, C.c_void_p, C.POINTER(C.c_int), C.c_void_p]
    lib.hylu_plan_save.argtypes = [H, C.c_void_p, C.POINTER(C.c_int64)]
    lib.hylu_plan_load.argtypes = [C.c_void_p, C.c_int64, C.POINTER(Options), C.POINTER(H)]
    _lib = lib
    return lib


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise HyluError(rc, where)
    return rc


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def default_options(**kw) -> Options:
    o = Options()
    load().hylu_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _host_csr(n, rowptr, col, vals=None, what="hylu_analyze"):
    """Host CSR arrays as the C ABI reads them (lengths n + 1, nnz, nnz)."""
    n = int(n)
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    if n < 0 or rowptr.ndim != 1 or len(rowptr) != n + 1:
        raise ValueError(f"{what}: rowptr must hold n + 1 = {n + 1} entries")
    nnz = int(rowptr[-1])
    if len(col) != nnz:
        raise ValueError(f"{what}: col must hold rowptr[n] = {nnz} entries, got {len(col)}")
    if vals is not None:
        vals = np.ascontiguousarray(vals, dtype=np.float64)
        if len(vals) != nnz:
            raise ValueError(f"{what}: vals must hold rowptr[n] = {nnz} entries, got {len(vals)}")
    return n, rowptr, col, vals


def hylu_analyze(n, rowptr, col, vals=None, user_perm=None, opt: Options | None = None) -> int:
    n, rowptr, col, vals = _host_csr(n, rowptr, col, vals)
    if user_perm is not None:
        user_perm = np.ascontiguousarray(user_perm, dtype=np.int32)
        if len(user_perm) != n:
            raise ValueError(f"hylu_analyze: user_perm must hold n = {n} entries")
    h = C.c_void_p()
    rc = load().hylu_analyze(int(n), int(rowptr[-1]), rowptr, col, _ptr(vals), _ptr(user_perm),
                             C.byref(opt) if opt is not None else None, C.byref(h))
    _check(rc, "hylu_analyze")
    return h.value


def hylu_factor(h: int, d_vals: int, stream: int = 0) -> int:
    return _check(load().hylu_factor(h, d_vals, stream), "hylu_factor")


def hylu_refactor(h: int, d_vals: int, stream: int = 0) -> int:
    return _check(load().hylu_refactor(h, d_vals, stream), "hylu_refactor")


def hylu_solve(h: int, d_b: int, d_x: int, nrhs: int, ld: int, stream: int = 0) -> int:
    return _check(load().hylu_solve(h, d_b, d_x, nrhs, ld, stream), "hylu_solve")


def hylu_solve_transpose(h: int, d_b: int, d_x: int, nrhs: int, ld: int, stream: int = 0) -> int:
    return _check(load().hylu_solve_transpose(h, d_b, d_x, nrhs, ld, stream), "hylu_solve_transpose")


def hylu_get_info(h: int) -> Info:
    info = Info()
    _check(load().hylu_get_info(h, C.byref(info)), "hylu_get_info")
    return info


def hylu_export_perm(h: int, n: int, nnodes: int):
    rp = np.empty(n, np.int32)
    cp = np.empty(n, np.int32)
    dr = np.empty(n, np.float64)
    dc = np.empty(n, np.float64)
    sn = np.empty(nnodes + 1, np.int32)
    _check(load().hylu_export_perm(h, _ptr(rp), _ptr(cp), _ptr(dr), _ptr(dc), _ptr(sn)), "hylu_export_perm")
    return rp, cp, dr, dc, sn


def hylu_export_pattern(h: int, n: int, nnz_store: int):
    rp = np.empty(n + 1, np.int64)
    ci = np.empty(nnz_store, np.int32)
    _check(load().hylu_export_pattern(h, _ptr(rp), _ptr(ci)), "hylu_export_pattern")
    return rp, ci


def hylu_export_schedule(h: int, n: int, ntasks: int, nheavy: int):
    order = np.empty(ntasks, np.int32)
    heavy = np.empty(max(nheavy, 0), np.int32)
    task_node = np.empty(ntasks - n, np.int32)
    _check(load().hylu_export_schedule(h, _ptr(order), _ptr(heavy), _ptr(task_node)), "hylu_export_schedule")
    return order, heavy, task_node


def hylu_export_factors(h: int, n: int, nnz_store: int):
    v = np.empty(nnz_store, np.float64)
    piv = np.empty(n, np.int32)
    _check(load().hylu_export_factors(h, _ptr(v), _ptr(piv)), "hylu_export_factors")
    return v, piv


def hylu_destroy(h: int) -> None:
    if h:
        load().hylu_destroy(h)


def hylu_launch_count() -> int:
    return int(load().hylu_launch_count())


def hylu_measure_fp64_peak(stream: int = 0) -> float:
    g = C.c_double()
    _check(load().hylu_measure_fp64_peak(C.byref(g), stream), "hylu_measure_fp64_peak")
    return g.value


GEMM_PLAN_ARRAYS = (
    ("gd_node", "ngd"), ("gd_Kp", "ngd"), ("gd_Mp", "ngd"), ("gd_a_off", "ngd"), ("gd_ntask", "ngd"),
    ("pair_gd", "npair"), ("pair_src", "npair"), ("pair_u0", "npair"), ("pair_len", "npair"),
    ("pair_jr", "npair"), ("pair_nj", "npair"), ("pair_need", "npair"), ("pair_x_off", "npair"),
    ("xmap", "nxmap"), ("gd_slot", "nl"), ("task_pair", "ntask"), ("task_mt", "ntask"), ("task_jt", "ntask"),
    ("task_level", "ntask"), ("row_order", "norder"), ("diag_row", "ndiag"), ("walk_level", "n"),
    ("diag_level", "n"))


def hylu_export_gemm_plan(h: int, min_rows: int, n: int) -> dict:
    """The tensor-core sup-sup tables for gemm_min_rows = min_rows, as a dict
    of int64 arrays (empty arrays when no node qualifies)."""
    lib = load()
    ln = C.c_int64(0)
    _check(lib.hylu_export_gemm_plan(h, int(min_rows), None, C.byref(ln)), "hylu_export_gemm_plan")
    buf = np.zeros(ln.value, np.int64)
    _check(lib.hylu_export_gemm_plan(h, int(min_rows), buf.ctypes.data, C.byref(ln)), "hylu_export_gemm_plan")
    names = ("ngd", "npair", "nxmap", "ntask", "ndiag", "norder", "levels", "nl", "min_src", "a_elems")
    cnt = dict(zip(names, (int(v) for v in buf[:10])))
    cnt["n"] = int(n)
    out = dict(cnt)
    pos = 10
    for name, size in GEMM_PLAN_ARRAYS:
        m = cnt[size] if cnt["ngd"] else 0
        out[name] = buf[pos:pos + m]
        pos += m
    return out


def hylu_export_solve_segments(h: int, backward: bool, max_rows: int) -> dict:
    """Bulk-sequential partition of a substitution (see include/hylu.h): the
    bulk claim list `task`, per segment `meta` (instance, first level, last
    level) and `seg_off`, per level `lvl_row` / `lvl_node`, `rows`, `snodes`,
    and the forward long rows' chunks (`chunk_row`, `chunk_a`, `chunk_b`,
    `chunk_level`, `row_chunk_off`)."""
    lib = load()
    ln = C.c_int64(0)
    _check(lib.hylu_export_solve_segments(h, int(bool(backward)), int(max_rows), None, C.byref(ln)),
           "hylu_export_solve_segments")
    buf = np.zeros(ln.value, np.int32)
    _check(lib.hylu_export_solve_segments(h, int(bool(backward)), int(max_rows), buf.ctypes.data, C.byref(ln)),
           "hylu_export_solve_segments")
    nt, ns, nl, nr, nn, nc = (int(v) for v in buf[:6])
    pos = 6
    n1 = len(buf) - pos - (nt + 3 * ns + ns + 1 + 2 * (nl + 1) + nr + nn + 4 * nc)   # n + 1
    out = {}
    for name, m in (("task", nt), ("meta", 3 * ns), ("seg_off", ns + 1), ("lvl_row", nl + 1),
                    ("lvl_node", nl + 1), ("rows", nr), ("snodes", nn), ("chunk_row", nc), ("chunk_a", nc),
                    ("chunk_b", nc), ("chunk_level", nc), ("row_chunk_off", n1)):
        out[name] = buf[pos:pos + m].copy()
        pos += m
    out["meta"] = out["meta"].reshape(-1, 3)
    return out


def hylu_debug_gemm(h: int, npair: int, ngd: int, n: int) -> dict:
    """Counters of the tensor-core sup-sup path after a factorization."""
    out = {"pair_cnt": np.zeros(npair, np.int32), "gd_done": np.zeros(ngd, np.int32),
           "walk_done": np.zeros(n, np.int32), "status": np.zeros(16, np.int32)}
    nb = C.c_int32(0)
    prog = np.zeros(4 * 4096, np.int32)
    _check(load().hylu_debug_gemm(h, *(out[k].ctypes.data for k in ("pair_cnt", "gd_done", "walk_done", "status")),
                                  prog.ctypes.data, C.byref(nb)), "hylu_debug_gemm")
    out["block_prog"] = prog[:4 * nb.value].reshape(-1, 4)
    return out


def hylu_split_gemm(d_a: int, d_b: int, d_c: int, m: int, n: int, k: int, lda: int, ldb: int, ldc: int,
                    nsplit: int = 3, stream: int = 0) -> int:
    """C -= A B on the tensor-core tile engine (FP32 arrays split into BF16
    terms; see include/hylu.h)."""
    return _check(load().hylu_split_gemm(d_a, d_b, d_c, m, n, k, lda, ldb, ldc, nsplit, stream),
                  "hylu_split_gemm")


def hylu_solve_static(h: int, d_b: int, d_x: int, stream: int = 0) -> int:
    """Allocation-free substitution for one right-hand side (see include/hylu.h)."""
    return _check(load().hylu_solve_static(h, d_b, d_x, stream), "hylu_solve_static")


def hylu_debug_trace(h: int, n: int):
    out = np.empty(4 * n, np.uint64)
    _check(load().hylu_debug_trace(h, _ptr(out)), "hylu_debug_trace")
    return out.reshape(n, 4)


def hylu_grad_values(h: int, d_lam: int, d_x: int, d_dvals: int, nrhs: int, ld: int, stream: int = 0) -> int:
    return _check(load().hylu_grad_values(h, d_lam, d_x, d_dvals, nrhs, ld, stream), "hylu_grad_values")


def hylu_analyze_batch(systems, nsets: int, opt: Options | None = None) -> int:
    """systems: list of (n, rowptr, col, vals) host arrays."""
    k = len(systems)
    ns = np.array([int(s[0]) for s in systems], np.int32)
    keep = []
    rps = (C.c_void_p * k)()
    cis = (C.c_void_p * k)()
    vls = (C.c_void_p * k)()
    for q, (n, rp, ci, v) in enumerate(systems):
        _, rp, ci, v = _host_csr(n, rp, ci, v, f"hylu_analyze_batch system {q}")
        keep += [rp, ci, v]
        rps[q] = rp.ctypes.data
        cis[q] = ci.ctypes.data
        vls[q] = None if v is None else v.ctypes.data
    h = C.c_void_p()
    rc = load().hylu_analyze_batch(k, ns.ctypes.data_as(C.c_void_p), C.cast(rps, C.c_void_p),
                                   C.cast(cis, C.c_void_p), C.cast(vls, C.c_void_p), int(nsets),
                                   C.byref(opt) if opt is not None else None, C.byref(h))
    _check(rc, "hylu_analyze_batch")
    return h.value


def hylu_batch_layout(h: int, ninst: int):
    rb = np.empty(ninst, np.int32)
    vb = np.empty(ninst, np.int64)
    tot = C.c_int32()
    _check(load().hylu_batch_layout(h, _ptr(rb), _ptr(vb), C.byref(tot)), "hylu_batch_layout")
    return rb, vb, tot.value


def hylu_graph_capture(h: int, d_vals: int, d_b: int, d_x: int, nrhs: int, ld: int, corrections: int = 0,
                       stream: int = 0) -> int:
    return _check(load().hylu_graph_capture(h, d_vals, d_b, d_x, nrhs, ld, corrections, stream),
                  "hylu_graph_capture")


def hylu_graph_launch(h: int, stream: int = 0) -> int:
    return _check(load().hylu_graph_launch(h, stream), "hylu_graph_launch")


def hylu_plan_save(h: int) -> bytes:
    """The handle's analysis as a byte image (see include/hylu.h)."""
    lib = load()
    need = C.c_int64(0)
    _check(lib.hylu_plan_save(h, None, C.byref(need)), "hylu_plan_save")
    buf = C.create_string_buffer(max(need.value, 1))
    size = C.c_int64(need.value)
    _check(lib.hylu_plan_save(h, buf, C.byref(size)), "hylu_plan_save")
    return buf.raw[:size.value]


def hylu_plan_load(image: bytes, opt: Options | None = None) -> int:
    """A new handle from a byte image written by hylu_plan_save."""
    data = bytes(image)
    buf = C.create_string_buffer(data, len(data))
    h = C.c_void_p()
    _check(load().hylu_plan_load(buf, len(data), C.byref(opt) if opt is not None else None, C.byref(h)),
           "hylu_plan_load")
    return h.value


def hylu_tune(h: int, d_vals: int, stream: int = 0) -> int:
    b = C.c_int()
    _check(load().hylu_tune(h, d_vals, C.byref(b), stream), "hylu_tune")
    return b.value
