"""CPU FP64 oracle for HYLU's numeric factorization and substitution.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports or links this package, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, one step of the method at a
time; see the comments there for the paper sections each step follows).  This
module compiles it with gcc and wraps it with ctypes; it adds no arithmetic of
its own beyond array marshalling.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

# sqrt(eps_f64): relative small-pivot threshold (a reading: the paper names
# pivot perturbation but gives no threshold)
TAU_REL = 1.4901161193847656e-08


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, portable flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.c_void_p
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
    lib.or_new.restype = P
    lib.or_new.argtypes = [C.c_int]
    lib.or_free.argtypes = [P]
    lib.or_build_ahat.argtypes = [P, i64p, i32p, f64p, i32p, i32p, f64p, f64p]
    lib.or_symbolic.argtypes = [P]
    lib.or_supernodes.argtypes = [P, C.c_int]
    lib.or_pad.argtypes = [P]
    lib.or_factor.argtypes = [P, C.c_double]
    lib.or_solve.argtypes = [P, i32p, i32p, f64p, f64p, f64p, f64p]
    lib.or_solve_transpose.argtypes = [P, i32p, i32p, f64p, f64p, f64p, f64p]
    lib.or_backward_error.restype = C.c_double
    lib.or_backward_error.argtypes = [C.c_int, i64p, i32p, f64p, f64p, f64p, C.c_void_p]
    lib.or_solve_refine.argtypes = [P, i64p, i32p, f64p, i32p, i32p, f64p, f64p, f64p, f64p,
                                    C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double)]
    for nm, rt in (("or_f_nnz", C.c_int64), ("or_p_nnz", C.c_int64), ("or_nsn", C.c_int),
                   ("or_nperturb", C.c_int), ("or_tau", C.c_double), ("or_n", C.c_int),
                   ("or_flops_unpadded", C.c_double), ("or_flops_padded", C.c_double)):
        getattr(lib, nm).restype = rt
        getattr(lib, nm).argtypes = [P]
    lib.or_get_ahat.argtypes = [P, i64p, i32p, f64p]
    lib.or_get_f.argtypes = [P, i64p, i32p]
    lib.or_get_sn.argtypes = [P, i32p]
    lib.or_get_p.argtypes = [P, i64p, i32p]
    lib.or_get_factor.argtypes = [P, f64p, i32p, f64p]
    _lib = lib
    return lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Pattern:
    rowptr: np.ndarray
    col: np.ndarray


class Oracle:
    """One oracle factorization of A under given preprocessing outputs.

    ``rowperm``/``colperm`` map new index -> original index; ``dr``/``dc`` are
    indexed by original row/column (Sec. 2.1 static pivoting and scaling)."""

    def __init__(self, n, rowptr, col, val, rowperm=None, colperm=None, dr=None, dc=None,
                 sn_max: int = 256, tau_rel: float = TAU_REL, numeric: bool = True):
        lib = _load()
        self.n = int(n)
        self.A = (_i64(rowptr), _i32(col), _f64(val))
        ident = np.arange(self.n, dtype=np.int32)
        self.rowperm = _i32(ident if rowperm is None else rowperm)
        self.colperm = _i32(ident if colperm is None else colperm)
        self.dr = _f64(np.ones(self.n) if dr is None else dr)
        self.dc = _f64(np.ones(self.n) if dc is None else dc)
        self._c = lib.or_new(self.n)
        if lib.or_build_ahat(self._c, *self.A, self.rowperm, self.colperm, self.dr, self.dc) != 0:
            raise ValueError("bad permutation")
        lib.or_symbolic(self._c)
        lib.or_supernodes(self._c, int(sn_max))
        lib.or_pad(self._c)
        self.nperturb = None
        if numeric:
            self.refactor(tau_rel)

    def refactor(self, tau_rel: float = TAU_REL):
        r = _load().or_factor(self._c, float(tau_rel))
        if r < 0:
            raise RuntimeError("padded pattern is not closed under the elimination")
        self.nperturb = r
        return r

    def __del__(self):
        if getattr(self, "_c", None) and _lib is not None:
            _lib.or_free(self._c)
            self._c = None

    # ----------------------------------------------------------- outputs
    @property
    def ahat(self):
        lib = _load()
        nnz = int(self.A[0][-1])
        rp = np.empty(self.n + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        v = np.empty(nnz, np.float64)
        lib.or_get_ahat(self._c, rp, ci, v)
        return rp, ci, v

    @property
    def unpadded(self) -> Pattern:
        lib = _load()
        rp = np.empty(self.n + 1, np.int64)
        ci = np.empty(lib.or_f_nnz(self._c), np.int32)
        lib.or_get_f(self._c, rp, ci)
        return Pattern(rp, ci)

    @property
    def padded(self) -> Pattern:
        lib = _load()
        rp = np.empty(self.n + 1, np.int64)
        ci = np.empty(lib.or_p_nnz(self._c), np.int32)
        lib.or_get_p(self._c, rp, ci)
        return Pattern(rp, ci)

    @property
    def sn_start(self) -> np.ndarray:
        lib = _load()
        s = np.empty(lib.or_nsn(self._c) + 1, np.int32)
        lib.or_get_sn(self._c, s)
        return s

    @property
    def flops(self) -> tuple[float, float]:
        lib = _load()
        return lib.or_flops_unpadded(self._c), lib.or_flops_padded(self._c)

    @property
    def tau(self) -> float:
        return _load().or_tau(self._c)

    def factors(self):
        """(values on the padded pattern, piv[position] = label, pivots u_ii)."""
        lib = _load()
        v = np.empty(lib.or_p_nnz(self._c), np.float64)
        piv = np.empty(self.n, np.int32)
        ud = np.empty(self.n, np.float64)
        lib.or_get_factor(self._c, v, piv, ud)
        return v, piv, ud

    # ------------------------------------------------------------ solves
    def solve(self, b):
        x = np.empty(self.n)
        _load().or_solve(self._c, self.rowperm, self.colperm, self.dr, self.dc, _f64(b), x)
        return x

    def solve_transpose(self, g):
        y = np.empty(self.n)
        _load().or_solve_transpose(self._c, self.rowperm, self.colperm, self.dr, self.dc, _f64(g), y)
        return y

    def solve_refine(self, b, tol: float = 1e-12, maxit: int = 10, force: bool = False):
        x = np.empty(self.n)
        be = C.c_double()
        it = _load().or_solve_refine(self._c, *self.A, self.rowperm, self.colperm, self.dr, self.dc,
                                     _f64(b), x, float(tol), int(maxit), int(force), C.byref(be))
        return x, it, be.value


def backward_error(n, rowptr, col, val, x, b) -> float:
    """||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) in FP64."""
    return _load().or_backward_error(int(n), _i64(rowptr), _i32(col), _f64(val), _f64(x), _f64(b), None)


def dense_factors(o: Oracle):
    """Dense (L, U, piv) in POSITION order from the stored factors: L unit
    lower, U upper, with Ahat[:, piv] = L @ U.  For small n only."""
    n = o.n
    P = o.padded
    v, piv, _ = o.factors()
    sn = o.sn_start
    end_of = np.empty(n, np.int64)
    for s in range(len(sn) - 1):
        end_of[sn[s]:sn[s + 1]] = sn[s + 1] - 1
    pinv = np.empty(n, np.int64)
    pinv[piv] = np.arange(n)
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for q in range(P.rowptr[i], P.rowptr[i + 1]):
            c = int(P.col[q])
            if c < i:
                L[i, c] = v[q]
            else:
                p = c if c <= end_of[i] else pinv[c]
                U[i, p] = v[q]
    return L, U, piv


def csr_dense(n, rowptr, col, val):
    a = np.zeros((n, n))
    for i in range(n):
        a[i, col[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
    return a
