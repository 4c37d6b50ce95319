"""Host-side checks that need no GPU: the C ABI library loads and exports
every entry point declared in include/hylu.h; preprocessing (Sec. 2.1) is
pinned by brute force and by the properties the paper states; the symbolic
pattern, supernode partition and flop count of the library equal the
oracle's bit for bit; malformed input returns the documented error codes."""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
from paper_2509_07690_gb300 import capi, synth
from paper_2509_07690_gb300.solver import Solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    header = open(os.path.join(ROOT, "include", "hylu.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t)\s+(hylu_\w+)\s*\(", header, re.M))
    assert {"hylu_analyze", "hylu_factor", "hylu_refactor", "hylu_solve",
            "hylu_solve_transpose"} <= declared
    lib = capi.load()
    for name in sorted(declared):
        assert hasattr(lib, name), name


def test_binding_constants_match_the_header():
    """Every #define HYLU_* of include/hylu.h has the same value in the binding."""
    header = open(os.path.join(ROOT, "include", "hylu.h")).read()
    defines = re.findall(r"^#define\s+(HYLU_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", header, re.M)
    assert {name for name, _ in defines} == {k for k in dir(capi) if k.startswith("HYLU_")}
    for name, value in defines:
        assert getattr(capi, name) == int(value), name
    assert capi.ERRORS[-9] == "HYLU_ERR_TOO_LARGE" and len(capi.ERRORS) == 9


def _dense_csr(a):
    r, c = np.nonzero(a)
    return synth.from_coo(a.shape[0], r, c, a[r, c])


# ------------------------------------------------------------------ MWM
def _scaled(s, A):
    rp, cp, dr, dc, _ = s.export_perm()
    a = A.todense()
    return (dr[:, None] * a * dc[None, :])[np.ix_(rp, cp)], rp, cp


@pytest.mark.parametrize("seed", range(25))
def test_matching_maximizes_product_brute_force(seed):
    """Sec. 2.1: the static pivot maximizes the product of the matched
    magnitudes; brute force over all n! permutations for n <= 7."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 8))
    a = np.where(rng.random((n, n)) < 0.6, rng.uniform(-3, 3, (n, n)), 0.0)
    a[np.arange(n), rng.permutation(n)] = rng.uniform(0.1, 2.0, n)   # a perfect matching exists
    A = _dense_csr(a)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=2)
    rp, cp, _, _, _ = s.export_perm()
    got = np.prod([abs(a[rp[i], cp[i]]) for i in range(n)])
    best = max(np.prod([abs(a[i, p[i]]) for i in range(n)]) for p in itertools.permutations(range(n)))
    assert got == pytest.approx(best, rel=1e-12)
    s.close()


@pytest.mark.parametrize("seed", range(10))
def test_scaling_unit_diagonal_bounded_offdiagonal(seed):
    """Sec. 2.1: after static pivoting and scaling the diagonal is +-1 and
    every other entry lies in [-1, 1]."""
    rng = np.random.default_rng(50 + seed)
    n = int(rng.integers(20, 120))
    a = np.where(rng.random((n, n)) < 0.1, rng.lognormal(0, 2, (n, n)) * rng.choice([-1, 1], (n, n)), 0.0)
    a[np.arange(n), rng.permutation(n)] = rng.lognormal(0, 2, n)
    A = _dense_csr(a)
    s = Solver(A.n, A.rowptr, A.col, A.val)
    ah, _, _ = _scaled(s, A)
    np.testing.assert_allclose(np.abs(np.diag(ah)), 1.0, rtol=1e-12)
    assert np.abs(ah).max() <= 1.0 + 1e-12
    s.close()


def test_matching_recovers_row_permutation():
    rng = np.random.default_rng(3)
    n = 300
    A = synth.grid5(10)
    a = A.todense()
    perm = rng.permutation(a.shape[0])
    B = _dense_csr(a[perm])
    s = Solver(B.n, B.rowptr, B.col, B.val, ordering=2)
    rp, cp, _, _, _ = s.export_perm()
    assert np.array_equal(perm[rp], cp)       # row of A that lands on column k is column k's row
    s.close()


def test_diagonally_dominant_gives_identity_matching():
    for A in (synth.grid5(12), synth.circuit(2000, seed=3)):
        s = Solver(A.n, A.rowptr, A.col, A.val)
        rp, cp, _, _, _ = s.export_perm()
        assert np.array_equal(rp, cp)
        s.close()


# ------------------------------------------------------------ orderings
@pytest.mark.parametrize("ordering", [0, 1])
def test_orderings_are_permutations_and_reduce_fill(ordering):
    for A in (synth.grid5(32), synth.aniso9(24), synth.convdiff3d(10)):
        s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering)
        rp, cp, _, _, _ = s.export_perm()
        assert np.array_equal(np.sort(cp), np.arange(A.n))
        nat = Solver(A.n, A.rowptr, A.col, A.val, ordering=2)
        assert s.info.nnz_lu < nat.info.nnz_lu
        s.close()
        nat.close()


ORDERING_QUALITY = [
    ("grid5_64", lambda: synth.grid5(64)),
    ("aniso_32", lambda: synth.aniso9(32)),
    ("convdiff_12", lambda: synth.convdiff3d(12)),
    ("circuit_3000", lambda: synth.circuit(3000, seed=12)),
    ("circuit_20000", lambda: synth.circuit(20000, seed=3)),
]


@pytest.mark.parametrize("name,make", ORDERING_QUALITY, ids=[c[0] for c in ORDERING_QUALITY])
def test_ordering_fill_close_to_superlu_mmd(name, make):
    """Fill of the AMD and nested dissection orderings against an independent
    library ordering: SuperLU's multiple minimum degree on A^T + A (scipy
    splu, diagonal pivots, symmetric mode), |L| + |U| counted with the
    diagonal once.  AMD stays within 1.1x of it; nested dissection within
    1.35x, circuit matrices included (their hub rows are ordered last, as
    AMD orders them)."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    import scipy.sparse as sp
    A = make()
    M = sp.csc_matrix(sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n)))
    lu = sla.splu(M, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0, options={"SymmetricMode": True})
    mmd = lu.L.nnz + lu.U.nnz - A.n
    for ordering, bound in ((0, 1.1), (1, 1.35)):
        s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering)
        assert s.info.nnz_lu <= bound * mmd, (ordering, s.info.nnz_lu, mmd)
        s.close()


def _estimate(info):
    return max(info.flops / 1.06e12, info.factor_levels * 21e-6)


@pytest.mark.parametrize("name,make", [("grid5_32", lambda: synth.grid5(32)),
                                       ("circuit_20000", lambda: synth.circuit(20000, seed=3)),
                                       ("convdiff_12", lambda: synth.convdiff3d(12)),
                                       ("circuit_100k", lambda: synth.workload("circuit_100k"))])
def test_auto_ordering_keeps_the_lower_estimate(name, make):
    """HYLU_ORDER_AUTO analyses under AMD and nested dissection and keeps the
    plan with the lower estimated factorization time (flops at the FP64 rate
    against the dependency chain); the kept plan is the one that ordering
    gives on its own."""
    A = make()
    views, est = {}, {}
    for o in (0, 1):
        s = Solver(A.n, A.rowptr, A.col, A.val, ordering=o)
        assert s.info.ordering == o
        est[o] = _estimate(s.info)
        v = _plan_views(s.h)
        views[o] = v
        s.close()
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=4)
    want = 1 if est[1] < est[0] else 0
    assert s.info.ordering == want
    v = _plan_views(s.h)
    _same_views(views[want], v)
    s.close()
    if name == "circuit_100k":
        assert want == 1                                 # the shallower chain wins


def test_analysis_phase_times():
    """The four phase times (matching, ordering, symbolic and schedules,
    value map) are non-negative and add up to the analysis time."""
    for A, o in ((synth.circuit(5000, seed=1), 0), (synth.convdiff3d(12), 1), (synth.grid5(3), 2)):
        s = Solver(A.n, A.rowptr, A.col, A.val, ordering=o)
        ph = list(s.info.analyze_phase_ms)
        assert min(ph) >= 0.0 and s.info.analyze_ms > 0.0
        assert abs(sum(ph) - s.info.analyze_ms) <= 0.05 * s.info.analyze_ms + 0.05
        s.close()


def test_ordering_reported_and_checked():
    A = synth.grid5(10)
    for o in (0, 1, 2):
        s = Solver(A.n, A.rowptr, A.col, A.val, ordering=o)
        assert s.info.ordering == o
        s.close()
    s = Solver(A.n, A.rowptr, A.col, A.val, np.arange(A.n, dtype=np.int32)[::-1].copy(), ordering=3)
    assert s.info.ordering == 3
    s.close()
    for bad in (-1, 5):
        with pytest.raises(capi.HyluError) as e:
            capi.hylu_analyze(A.n, A.rowptr, A.col, A.val, None, capi.default_options(ordering=bad))
        assert e.value.code == -1
    from paper_2509_07690_gb300.solver import BatchSolver
    mats = [synth.grid5(6), synth.circuit(300, seed=4)]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], 1, ordering=1)
    assert bs.info.ordering == 1
    bs.close()
    # AUTO inside a batch: each system keeps its own better plan; the batch
    # reports the common choice, or AUTO when the systems chose differently
    mats = [synth.grid5(6), synth.circuit(300, seed=4), synth.circuit(2500, seed=9), synth.convdiff3d(6)]
    picks = []
    for m in mats:
        s = Solver(m.n, m.rowptr, m.col, m.val, ordering=4)
        picks.append(s.info.ordering)
        s.close()
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], 2, ordering=4)
    assert bs.info.ordering == (picks[0] if len(set(picks)) == 1 else 4)
    bs.close()


def test_nested_dissection_fill_grows_slowly_on_grids():
    """2D grids: nested dissection fill grows like n log n, not n^1.5."""
    fills = []
    for k in (32, 64, 128):
        A = synth.grid5(k)
        s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1)
        fills.append(s.info.nnz_lu / (A.n * np.log2(A.n)))
        s.close()
    assert fills[-1] < 2.0 * fills[0]


# --------------------------------------------- pattern parity on the host
CASES = [
    ("grid5_16", lambda: synth.grid5(16), {}),
    ("grid5_64", lambda: synth.grid5(64), {}),
    ("circuit_3000", lambda: synth.circuit(3000, seed=12), {}),
    ("convdiff_10_nd", lambda: synth.convdiff3d(10), {"ordering": 1}),
    ("aniso_32_nd", lambda: synth.aniso9(32), {"ordering": 1}),
    ("convdiff_8_sn7", lambda: synth.convdiff3d(8), {"ordering": 1, "sn_max": 7}),
]


def _kernel_split(o):
    """The padded flops of the oracle's pattern by kernel: every L entry of
    row i in column k costs 1 + 2 (|U(k,:)| - 1) (unpadded U row length);
    a standalone source is row-row, a supernode source sup-row into a
    standalone row and sup-sup into a supernode row; the columns of a row's
    own supernode before it are the in-supernode factorization."""
    sn = np.asarray(o.sn_start)
    size = np.diff(sn)
    node = np.repeat(np.arange(len(size)), size)
    urp, uci = o.unpadded.rowptr, o.unpadded.col
    n = len(node)
    ulen = np.array([np.count_nonzero(uci[urp[k]:urp[k + 1]] >= k) for k in range(n)], dtype=np.int64)
    g = 1 + 2 * (ulen - 1)
    prp, pci = o.padded.rowptr, o.padded.col
    rr = sr = ss = ins = 0
    for i in range(n):
        r = sn[node[i]]
        cols = pci[prp[i]:prp[i + 1]]
        lc = cols[cols < r]
        from_sn = size[node[lc]] > 1
        rr += int(g[lc[~from_sn]].sum())
        if size[node[i]] > 1:
            ss += int(g[lc[from_sn]].sum())
        else:
            sr += int(g[lc[from_sn]].sum())
        ins += int(g[r:i].sum())
    return rr, sr, ss, ins


@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_pattern_partition_flops_bit_exact(name, make, opts):
    A = make()
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc, sn_max=opts.get("sn_max", 256), numeric=False)
    prp, pci = s.export_pattern()
    assert np.array_equal(o.sn_start, sn)
    assert np.array_equal(o.padded.rowptr, prp) and np.array_equal(o.padded.col, pci)
    assert s.info.nnz_lu == len(o.unpadded.col)
    assert s.info.flops == o.flops[0] and s.info.flops_padded == o.flops[1]
    split = _kernel_split(o)
    assert sum(split) == o.flops[1]
    assert (s.info.flops_row_row, s.info.flops_sup_row, s.info.flops_sup_sup, s.info.flops_in_supernode) == split
    s.close()


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_pattern_parity_degenerate_sizes(n):
    """The smallest systems: the empty matrix has no supernode (partition
    [0]) and no flops; n = 1 is one standalone row.  Pattern, partition and
    flop count equal the oracle's bit for bit."""
    a = 3.0 * np.eye(n) + np.triu(np.ones((n, n)), 1) - 0.5 * np.tril(np.ones((n, n)), -2)
    A = _dense_csr(a)
    s = Solver(A.n, A.rowptr, A.col, A.val)
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc, numeric=False)
    prp, pci = s.export_pattern()
    assert np.array_equal(o.sn_start, sn) and sn[0] == 0 and sn[-1] == n
    if n == 0:
        assert list(sn) == [0]
    assert np.array_equal(o.padded.rowptr, prp) and np.array_equal(o.padded.col, pci)
    assert s.info.flops == o.flops[0] and s.info.flops_padded == o.flops[1]
    assert s.info.nnodes == len(sn) - 1
    s.close()


def _degenerate(kind):
    rng = np.random.default_rng(77)
    if kind == "diagonal":                 # every row standalone, no L, no U tail
        n = 500
        return synth.from_coo(n, np.arange(n), np.arange(n), rng.uniform(1, 2, n))
    if kind == "permutation":              # the matching must undo a row permutation
        n = 300
        p = rng.permutation(n)
        return synth.from_coo(n, p, np.arange(n), rng.uniform(1, 2, n) * rng.choice([-1, 1], n))
    if kind == "upper_dense":              # dense upper triangle
        n = 40
        r, c = np.triu_indices(n)
        return synth.from_coo(n, r, c, np.where(r == c, 5.0, rng.uniform(-1, 1, len(r))))
    if kind == "lower_bidiagonal":         # one chain of standalone rows
        n = 200
        r = np.concatenate([np.arange(n), np.arange(1, n)])
        c = np.concatenate([np.arange(n), np.arange(n - 1)])
        return synth.from_coo(n, r, c, np.concatenate([np.full(n, 3.0), np.full(n - 1, -1.0)]))
    if kind == "arrow_first":              # dense first row and column
        n = 120
        r = np.concatenate([np.arange(n), np.zeros(n - 1, int), np.arange(1, n)])
        c = np.concatenate([np.arange(n), np.arange(1, n), np.zeros(n - 1, int)])
        v = np.concatenate([np.full(n, 4.0), rng.uniform(-1, 1, 2 * (n - 1))])
        return synth.from_coo(n, r, c, v)
    raise KeyError(kind)


@pytest.mark.parametrize("ordering", [0, 1, 2])
@pytest.mark.parametrize("kind", ["diagonal", "permutation", "upper_dense", "lower_bidiagonal", "arrow_first"])
def test_pattern_parity_degenerate_structures(kind, ordering):
    """Structures at the edges of the method: a diagonal matrix, a row
    permutation of one, a dense triangle, a single chain and a dense first
    row and column, under AMD, nested dissection and the natural order.  The
    matching gives a zero-free diagonal, and the pattern, partition and flop
    count equal the oracle's bit for bit."""
    A = _degenerate(kind)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering)
    rp, cp, dr, dc, sn = s.export_perm()
    assert sorted(rp) == list(range(A.n)) and sorted(cp) == list(range(A.n))
    a = A.todense()
    assert np.all(a[rp, cp] != 0)                     # zero-free diagonal after static pivoting
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc, numeric=False)
    prp, pci = s.export_pattern()
    assert np.array_equal(o.sn_start, sn)
    assert np.array_equal(o.padded.rowptr, prp) and np.array_equal(o.padded.col, pci)
    assert s.info.flops == o.flops[0] and s.info.flops_padded == o.flops[1]
    if kind in ("diagonal", "permutation"):
        assert s.info.flops == 0.0 and s.info.nnz_lu == A.n
    s.close()


@pytest.mark.parametrize("seed", range(30))
def test_pattern_parity_random_unsymmetric(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(5, 90))
    a = np.where(rng.random((n, n)) < rng.uniform(0.02, 0.15), rng.uniform(-1, 1, (n, n)), 0.0)
    a[np.arange(n), np.arange(n)] += rng.uniform(1, 2, n)
    A = _dense_csr(a)
    user = rng.permutation(n).astype(np.int32)
    s = Solver(A.n, A.rowptr, A.col, A.val, user, ordering=3, static_pivot=0, sn_max=int(rng.integers(1, 9)))
    rp, cp, dr, dc, sn = s.export_perm()
    assert np.array_equal(cp, user) and np.array_equal(rp, user)
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, user, user, None, None, sn_max=s.opt.sn_max, numeric=False)
    prp, pci = s.export_pattern()
    assert np.array_equal(o.sn_start, sn)
    assert np.array_equal(o.padded.col, pci) and np.array_equal(o.padded.rowptr, prp)
    assert s.info.flops == o.flops[0]
    s.close()


@pytest.mark.parametrize("seed", range(20))
def test_nested_dissection_with_dense_vertices(seed):
    """Random sparse matrices with a few planted dense rows and columns under
    nested dissection (dense vertices set aside and ordered last) and AUTO:
    the ordering is a permutation with the dense vertices at its end, and the
    pattern, partition and flop count equal the oracle's."""
    rng = np.random.default_rng(2200 + seed)
    n = int(rng.integers(40, 400))
    a = np.where(rng.random((n, n)) < 4.0 / n, rng.uniform(-1, 1, (n, n)), 0.0)
    hubs = rng.choice(n, int(rng.integers(1, 5)), replace=False)
    for h in hubs:
        a[h, :] = np.where(rng.random(n) < 0.6, rng.uniform(-1, 1, n), a[h, :])
        a[:, h] = np.where(rng.random(n) < 0.6, rng.uniform(-1, 1, n), a[:, h])
    a[np.arange(n), np.arange(n)] = np.abs(a).sum(axis=1) + 1.0
    A = _dense_csr(a)
    for ordering in (1, 4):
        s = Solver(A.n, A.rowptr, A.col, A.val, ordering=ordering)
        rp, cp, dr, dc, sn = s.export_perm()
        assert sorted(cp) == list(range(n))
        if ordering == 1:
            # dense: degree in A + A^T (no diagonal) above max(16, min(2 sqrt(n), 10 x mean degree))
            pat = (a != 0) | (a.T != 0)
            np.fill_diagonal(pat, False)
            deg = pat.sum(axis=1)
            thr = max(16, int(min(2.0 * np.sqrt(n), 10.0 * deg.sum() / n)))
            dense = np.nonzero(deg > thr)[0]
            assert set(hubs.tolist()) <= set(dense.tolist())
            assert list(cp[n - len(dense):]) == sorted(dense.tolist())
        o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc, numeric=False)
        prp, pci = s.export_pattern()
        assert np.array_equal(o.sn_start, sn)
        assert np.array_equal(o.padded.rowptr, prp) and np.array_equal(o.padded.col, pci)
        assert s.info.flops == o.flops[0]
        s.close()


@pytest.mark.parametrize("seed", range(16))
def test_pattern_parity_chains_and_dense_rows(seed):
    """Dense diagonal blocks with one-sided couplings (long runs of rows whose
    U structures nest, cut by pruning and unsymmetry at odd places) followed by
    an arrowhead of dense rows and columns (rows dense over their whole range):
    the symbolic shortcuts for chains and dense rows give the oracle's sets."""
    rng = np.random.default_rng(1700 + seed)
    nb = int(rng.integers(2, 7))
    sizes = rng.integers(1, 24, nb)
    n0 = int(sizes.sum())
    h = int(rng.integers(1, 6))
    n = n0 + h
    a = np.zeros((n, n))
    off = 0
    for b in sizes:
        blk = np.where(rng.random((b, b)) < 0.8, rng.uniform(-1, 1, (b, b)), 0.0)
        a[off:off + b, off:off + b] = blk
        if off > 0:                      # one-sided coupling to an earlier block
            c = int(rng.integers(0, off))
            if rng.random() < 0.5:
                a[off + int(rng.integers(0, b)), c] = 0.5
            else:
                a[c, off + int(rng.integers(0, b))] = 0.5
        off += b
    for t in range(h):                  # arrowhead rows / columns, partly dense
        r = n0 + t
        a[r, :] = np.where(rng.random(n) < rng.uniform(0.3, 1.0), rng.uniform(-1, 1, n), 0.0)
        a[:, r] = np.where(rng.random(n) < rng.uniform(0.3, 1.0), rng.uniform(-1, 1, n), a[:, r])
    a[np.arange(n), np.arange(n)] += rng.uniform(2, 3, n)
    A = _dense_csr(a)
    perm = np.arange(n, dtype=np.int32)
    if seed % 2:                        # scramble the blocks' interiors, keep the arrow last
        perm[:n0] = rng.permutation(n0).astype(np.int32)
    s = Solver(A.n, A.rowptr, A.col, A.val, perm, ordering=3, static_pivot=0,
               sn_max=int(rng.choice([1, 3, 8, 256])))
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, perm, perm, None, None, sn_max=s.opt.sn_max, numeric=False)
    prp, pci = s.export_pattern()
    rp, cp, dr, dc, sn = s.export_perm()
    assert np.array_equal(o.sn_start, sn)
    assert np.array_equal(o.padded.col, pci) and np.array_equal(o.padded.rowptr, prp)
    assert s.info.nnz_lu == len(o.unpadded.col)
    assert s.info.flops == o.flops[0] and s.info.flops_padded == o.flops[1]
    s.close()


# ------------------------------------------------------------- errors
def test_error_codes():
    rp = np.array([0, 2, 3], np.int64)
    with pytest.raises(capi.HyluError) as e:          # unsorted columns
        capi.hylu_analyze(2, rp, np.array([1, 0, 1], np.int32), np.ones(3))
    assert e.value.code == -2
    with pytest.raises(capi.HyluError) as e:          # out of range
        capi.hylu_analyze(2, rp, np.array([0, 5, 1], np.int32), np.ones(3))
    assert e.value.code == -2
    with pytest.raises(capi.HyluError) as e:          # structurally singular: empty column 1
        capi.hylu_analyze(2, np.array([0, 1, 2], np.int64), np.array([0, 0], np.int32), np.ones(2))
    assert e.value.code == -3
    with pytest.raises(capi.HyluError) as e:          # bad user permutation
        capi.hylu_analyze(2, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32), np.ones(2),
                          np.array([0, 0], np.int32), capi.default_options(ordering=3))
    assert e.value.code == -1
    A = synth.grid5(4)
    for bad in (np.nan, np.inf, -np.inf):             # the matching needs finite values
        v = A.val.copy()
        v[3] = bad
        with pytest.raises(capi.HyluError) as e:
            capi.hylu_analyze(A.n, A.rowptr, A.col, v)
        assert e.value.code == -1
        h = capi.hylu_analyze(A.n, A.rowptr, A.col, v, None, capi.default_options(static_pivot=0))
        capi.hylu_destroy(h)                          # without static pivoting the values are not read
    h = capi.hylu_analyze(A.n, A.rowptr, A.col, A.val)
    with pytest.raises(capi.HyluError) as e:          # refactor before factor
        capi.hylu_refactor(h, 0, 0)
    assert e.value.code in (-1, -7)
    with pytest.raises(capi.HyluError) as e:          # solve before factor
        capi.hylu_solve(h, 1, 1, 1, A.n, 0)
    assert e.value.code == -7
    capi.hylu_destroy(h)


def test_binding_refuses_arrays_of_the_wrong_size_or_type():
    """Host arrays whose lengths disagree with n and rowptr[n], and tensors of
    another dtype, device or size, are refused before the library reads them
    (the C ABI takes plain pointers and trusts the sizes)."""
    torch = pytest.importorskip("torch")
    A = synth.grid5(4)
    with pytest.raises(ValueError):
        capi.hylu_analyze(A.n, A.rowptr[:-1], A.col, A.val)
    with pytest.raises(ValueError):
        capi.hylu_analyze(A.n, A.rowptr, A.col[:-1], A.val)
    with pytest.raises(ValueError):
        capi.hylu_analyze(A.n, A.rowptr, A.col, A.val[:-1])
    with pytest.raises(ValueError):
        capi.hylu_analyze(A.n, A.rowptr, A.col, A.val, np.arange(A.n - 1, dtype=np.int32),
                          capi.default_options(ordering=3))
    with pytest.raises(ValueError):
        capi.hylu_analyze_batch([(A.n, A.rowptr, A.col, A.val[:-2])], 1)
    with pytest.raises(capi.HyluError) as e:          # no values, but static pivoting wants them
        capi.hylu_analyze_batch([(A.n, A.rowptr, A.col, None)], 1)
    assert e.value.code == -1
    s = Solver(A.n, A.rowptr, A.col, A.val)
    with pytest.raises(TypeError):                    # host tensor
        s.factor(torch.from_numpy(A.val))
    with pytest.raises(TypeError):                    # host tensor, wrong dtype
        s.factor(torch.from_numpy(A.val).float())
    with pytest.raises(TypeError):
        s.solve(torch.zeros(A.n, dtype=torch.float64))
    with pytest.raises(TypeError):
        s.factor(A.val)
    s.close()


def test_solver_from_scipy_csr():
    """A scipy CSR matrix with unsorted column indices: the solver sorts a
    copy per row (values moved with their columns) and analyses the same
    pattern as the sorted CSR; a duplicate entry is refused."""
    sp = pytest.importorskip("scipy.sparse")
    A = synth.circuit(1500, seed=5)
    M = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    rng = np.random.default_rng(2)
    ind, dat = M.indices.copy(), M.data.copy()
    for i in range(A.n):                               # shuffle every row
        a, b = M.indptr[i], M.indptr[i + 1]
        o = rng.permutation(b - a)
        ind[a:b], dat[a:b] = ind[a:b][o], dat[a:b][o]
    U = sp.csr_matrix((dat, ind, M.indptr.copy()), shape=M.shape)
    assert not U.has_sorted_indices
    s = Solver.from_csr(U)
    ref = Solver(A.n, A.rowptr, A.col, A.val)
    assert np.array_equal(s.values, A.val)
    _same_views(_plan_views(s.h), _plan_views(ref.h))
    s.close()
    ref.close()
    D = sp.csr_matrix((np.array([1.0, 2.0, 3.0]), np.array([0, 0, 1]), np.array([0, 2, 3])), shape=(2, 2))
    with pytest.raises(capi.HyluError) as e:
        Solver.from_csr(D)
    assert e.value.code == -2
    with pytest.raises(ValueError):
        Solver.from_csr(sp.csr_matrix(np.ones((2, 3))))


# ------------------------------------------------------ empty system
def test_empty_system_returns_ok_without_device_work():
    """n = 0 is a valid, degenerate system: analysis gives an empty plan, and
    factorization, refactorization, both solves, the gradient scatter, the
    grid tuner and the exports return HYLU_OK with NULL device pointers and
    launch no kernel (none of these calls reaches the CUDA runtime, so this
    runs without a GPU).  A solve before the factorization is still refused."""
    rp = np.zeros(1, np.int64)
    ci = np.zeros(0, np.int32)
    h = capi.hylu_analyze(0, rp, ci, np.zeros(0))
    info = capi.hylu_get_info(h)
    assert (info.n, info.nnz_a, info.nnz_lu, info.nnz_store, info.nnodes) == (0, 0, 0, 0, 0)
    assert info.flops == 0.0 and info.flops_padded == 0.0
    with pytest.raises(capi.HyluError) as e:
        capi.hylu_solve(h, 0, 0, 1, 0, 0)
    assert e.value.code == -7
    l0 = capi.hylu_launch_count()
    assert capi.hylu_factor(h, 0, 0) == 0
    assert capi.hylu_refactor(h, 0, 0) == 0
    assert capi.hylu_solve(h, 0, 0, 1, 0, 0) == 0
    assert capi.hylu_solve(h, 0, 0, 3, 0, 0) == 0
    assert capi.hylu_solve_transpose(h, 0, 0, 2, 0, 0) == 0
    assert capi.hylu_grad_values(h, 0, 0, 0, 1, 0, 0) == 0
    assert capi.hylu_tune(h, 1, 0) == 1
    with pytest.raises(capi.HyluError) as e:          # nrhs must still be positive
        capi.hylu_solve(h, 0, 0, 0, 0, 0)
    assert e.value.code == -1
    assert capi.hylu_launch_count() == l0
    info = capi.hylu_get_info(h)
    assert info.device_status == 0 and info.nperturb == 0
    rowperm, colperm, dr, dc, sn = capi.hylu_export_perm(h, 0, info.nnodes)
    assert len(rowperm) == 0 and list(sn) == [0]
    prp, pci = capi.hylu_export_pattern(h, 0, 0)
    assert list(prp) == [0] and len(pci) == 0
    v, piv = capi.hylu_export_factors(h, 0, 0)
    assert len(v) == 0 and len(piv) == 0
    capi.hylu_destroy(h)
    A = synth.grid5(3)                                # a batch refuses an empty system
    with pytest.raises(capi.HyluError) as e:
        capi.hylu_analyze_batch([(A.n, A.rowptr, A.col, A.val), (0, rp, ci, np.zeros(0))], 1)
    assert e.value.code == -1


def test_empty_system_through_the_binding():
    """The handle wrapper passes empty tensors of an empty system through
    (shapes [0] and [nrhs, 0]) instead of reshaping by a zero width.  The
    tensors here are host tensors that report is_cuda, so the marshalling is
    checked without a GPU; no call reaches the device for n = 0."""
    torch = pytest.importorskip("torch")
    from types import SimpleNamespace

    class Tagged(torch.Tensor):
        @property
        def is_cuda(self):
            return True

    def dev(*shape):
        return torch.Tensor._make_subclass(Tagged, torch.zeros(*shape, dtype=torch.float64))

    st = SimpleNamespace(cuda_stream=0)
    s = Solver(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    l0 = capi.hylu_launch_count()
    assert s.factor(dev(0), stream=st) == 0
    x = s.solve(dev(0), stream=st)
    assert tuple(x.shape) == (0,)
    x = s.solve(dev(4, 0), dev(4, 0), stream=st, transpose=True)
    assert tuple(x.shape) == (4, 0)
    with pytest.raises(ValueError):                   # an empty system takes empty tensors
        s.solve(dev(3), stream=st)
    A = synth.grid5(4)                                # the solution may not overwrite b
    t = Solver(A.n, A.rowptr, A.col, A.val)
    b = dev(2, A.n)
    with pytest.raises(ValueError):
        t.solve(b, b, stream=st)
    with pytest.raises(ValueError):
        t.solve(b[0], b.view(-1)[5:5 + A.n], stream=st)
    t.close()
    assert capi.hylu_launch_count() == l0
    assert s.get_info().device_status == 0
    s.close()


# ------------------------------------------------ checkpoint of an analysis
# info fields that describe the plan (wall times are not part of it)
INFO_FIELDS = ["n", "nnz_a", "nnz_lu", "nnz_store", "nnodes", "nsupernodes", "rows_in_supernodes",
               "max_supernode", "ntasks", "flops", "flops_padded", "nheavy", "factor_levels",
               "fwd_levels", "bwd_levels", "flops_row_row", "flops_sup_row", "flops_sup_sup",
               "flops_in_supernode", "ordering"]


def _plan_views(h):
    """Everything the C ABI shows of a plan: sizes, preprocessing, pattern, schedule."""
    info = capi.hylu_get_info(h)
    views = [getattr(info, f) for f in INFO_FIELDS]
    views += list(capi.hylu_export_perm(h, info.n, info.nnodes))
    views += list(capi.hylu_export_pattern(h, info.n, info.nnz_store))
    views += list(capi.hylu_export_schedule(h, info.n, info.ntasks, info.nheavy))
    return views


def _same_views(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for byte in data:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


CHECKPOINT_CASES = [
    ("grid5_16", lambda: synth.grid5(16), {}),
    ("circuit_3000_heavy", lambda: synth.circuit(3000, seed=12), {"heavy_ratio": 1.0}),
    ("convdiff_8_nd_sn7", lambda: synth.convdiff3d(8), {"ordering": 1, "sn_max": 7}),
    ("aniso_24_nd", lambda: synth.aniso9(24), {"ordering": 1}),
    ("grid5_12_fp32", lambda: synth.grid5(12), {"precision": 1}),
    ("empty", lambda: synth.from_coo(0, [], [], []), {}),
]


@pytest.mark.parametrize("name,make,opts", CHECKPOINT_CASES, ids=[c[0] for c in CHECKPOINT_CASES])
def test_plan_checkpoint_round_trip(name, make, opts, tmp_path):
    """A saved analysis loads into a handle whose sizes, permutations,
    scalings, supernodes, padded pattern and schedules equal the original's,
    and saving the loaded handle gives the same bytes.  Numeric options given
    at load time change the options, not the plan."""
    A = make()
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    path = tmp_path / "plan.bin"
    image = s.save(path)
    assert path.read_bytes() == image
    t = Solver.load(path)
    assert (t.n, t.nnz) == (A.n, A.nnz)
    _same_views(_plan_views(s.h), _plan_views(t.h))
    assert t.info.analyze_ms == s.info.analyze_ms                 # the analysis it saves
    assert list(t.info.analyze_phase_ms) == list(s.info.analyze_phase_ms)
    assert t.save() == image
    u = Solver.load(image, precision=1, pivot_tau=1e-10, spin_limit=1 << 20)
    _same_views(_plan_views(s.h), _plan_views(u.h))
    for x in (s, t, u):
        x.close()


def test_analysis_on_concurrent_host_threads():
    """Separate handles on separate host threads (ctypes releases the GIL
    during the C calls, so the analyses overlap): every plan equals the one
    the same input gives when analysed alone."""
    import threading
    mats = [(synth.circuit(2500, seed=40 + q), {}) for q in range(3)] + \
           [(synth.convdiff3d(9), {"ordering": 1}), (synth.aniso9(20), {"ordering": 1})]

    def views(A, opts):
        s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
        v = _plan_views(s.h)
        s.close()
        return v

    alone = [views(A, o) for A, o in mats]
    got = [None] * len(mats)

    def work(q):
        for _ in range(3):
            got[q] = views(*mats[q])

    th = [threading.Thread(target=work, args=(q,)) for q in range(len(mats))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for q in range(len(mats)):
        _same_views(alone[q], got[q])


def test_plan_checkpoint_batch():
    """A batch handle's image keeps the block-diagonal plan and its layout."""
    from paper_2509_07690_gb300.solver import BatchSolver
    mats = [synth.circuit(300, seed=5), synth.grid5(6), synth.circuit(800, seed=6)]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], 2)
    image = bs.save()
    t = Solver.load(image)
    assert t.n == bs.n and t.nnz == bs.nnz
    _same_views(_plan_views(bs.h), _plan_views(t.h))
    lay_a = capi.hylu_batch_layout(bs.h, 6)
    lay_b = capi.hylu_batch_layout(t.h, 6)
    _same_views(lay_a, lay_b)
    assert t.save() == image
    with pytest.raises(TypeError):
        BatchSolver.load(image)
    bs.close()
    t.close()


def test_plan_checkpoint_rejects_damaged_images():
    """Truncated, altered and foreign images are refused with
    HYLU_ERR_PATTERN: the checksum catches altered bytes, and an image whose
    checksum was recomputed over inconsistent sizes fails the size checks.
    The options block is 84 bytes after the 16-byte header, so n sits at
    byte 100."""
    A = synth.grid5(8)
    s = Solver(A.n, A.rowptr, A.col, A.val)
    image = s.save()

    def code(img):
        with pytest.raises(capi.HyluError) as e:
            capi.hylu_plan_load(img)
        return e.value.code

    def resealed(body: bytes) -> bytes:
        return body + _fnv1a(body).to_bytes(8, "little")

    flipped = bytearray(image)
    flipped[len(image) // 2] ^= 0x40
    assert code(bytes(flipped)) == -2                  # altered byte
    assert code(image[:-1]) == -2                      # truncated
    assert code(image[:40]) == -2
    assert code(b"XYLUPLAN" + image[8:]) == -2          # foreign magic
    body = bytearray(image[:-8])
    body[8] = 4                                        # a later version
    assert code(resealed(bytes(body))) == -2
    body = bytearray(image[:-8])
    assert int.from_bytes(body[108:112], "little") == A.n
    body[108:112] = (A.n + 1).to_bytes(4, "little")    # n no longer fits the arrays
    assert code(resealed(bytes(body))) == -2
    h = capi.hylu_plan_load(resealed(image[:-8]))     # resealing alone changes nothing
    assert h
    capi.hylu_destroy(h)
    with pytest.raises(capi.HyluError) as e:
        capi.hylu_plan_load(image, capi.default_options(precision=2))
    assert e.value.code == -1
    with pytest.raises(capi.HyluError) as e:
        capi.hylu_plan_load(b"")
    assert e.value.code == -1
    s.close()


# ------------------------------------------------- heavy-row claim queue
def test_heavy_rows_selection():
    """Circuit hub rows (dense rows ordered last, most sources finished early)
    are picked for the factor kernel's heavy-row queue; nested-dissection top
    separators (sources finishing late) are not; ratio 0 switches it off and a
    smaller ratio never picks fewer rows."""
    A = synth.circuit(20000, seed=77)
    counts = {}
    for r in (0.0, 1.0, 32.0):
        s = Solver(A.n, A.rowptr, A.col, A.val, heavy_ratio=r)
        counts[r] = s.get_info().nheavy
        s.close()
    assert counts[0.0] == 0
    assert counts[32.0] > 0
    assert counts[1.0] >= counts[32.0]
    B = synth.convdiff3d(16)
    s = Solver(B.n, B.rowptr, B.col, B.val, ordering=1)
    assert s.get_info().nheavy == 0
    s.close()
    with pytest.raises(capi.HyluError) as e:
        capi.hylu_analyze(A.n, A.rowptr, A.col, A.val, None, capi.default_options(heavy_ratio=-1.0))
    assert e.value.code == -1


def test_batch_plan_counts_sum_over_instances():
    """The combined plan of a batch holds every instance (system x value set)
    as its own block: rows, stored entries, flops and factor-kernel tasks
    (rows plus supernode tail tasks) are the sums over the instances."""
    from paper_2509_07690_gb300 import BatchSolver
    mats = [synth.circuit(n, seed=600 + n) for n in (300, 1200, 2500)] + [synth.convdiff3d(8)]
    singles = [Solver(m.n, m.rowptr, m.col, m.val) for m in mats]
    nsets = 3
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], nsets)
    info = bs.get_info()
    assert info.n == nsets * sum(m.n for m in mats)
    assert info.nnz_store == nsets * sum(s.info.nnz_store for s in singles)
    assert info.flops == nsets * sum(s.info.flops for s in singles)
    assert info.ntasks == nsets * sum(s.info.ntasks for s in singles)
    assert info.ntasks > info.n or all(s.info.ntasks == s.info.n for s in singles)
    for s in singles:
        s.close()
    bs.close()
