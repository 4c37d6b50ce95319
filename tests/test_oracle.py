"""Pins for the CPU oracle against what the paper and the mathematics fix:
closed forms, brute force, textbook routines and invariants (no GPU)."""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2509_07690_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


def tridiag(n, lo=-1.0, d=2.0, up=-1.0):
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i); cols.append(i); vals.append(d)
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(lo)
        if i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(up)
    return synth.from_coo(n, rows, cols, vals)


def dense_csr(a):
    n = a.shape[0]
    r, c = np.nonzero(a)
    return synth.from_coo(n, r, c, a[r, c])


def random_sparse(n, density, rng, diag=True, dominant=False):
    a = np.where(rng.random((n, n)) < density, rng.uniform(-1, 1, (n, n)), 0.0)
    if diag:
        a[np.arange(n), np.arange(n)] = rng.uniform(0.5, 1.5, n) * np.where(rng.random(n) < .5, -1, 1)
    if dominant:
        a[np.arange(n), np.arange(n)] = np.sign(np.diag(a) + 1e-300) * (np.abs(a).sum(1) + 1)
    return a


def read_golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        out[k] = np.array([float(t) for t in v])
    return out


# ----------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [2, 5, 17, 64])
def test_laplacian1d_pivots_closed_form(n):
    """tridiag(-1, 2, -1), natural order, no scaling: u_kk = (k+1)/k and
    L(k+1, k) = -k/(k+1) (1-based), exact up to rounding."""
    A = tridiag(n)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val)
    L, U, piv = oracle.dense_factors(o)
    k = np.arange(1, n + 1)
    np.testing.assert_allclose(np.diag(U), (k + 1) / k, rtol=4 * n * EPS)
    np.testing.assert_allclose(np.diag(L, -1), -k[:-1] / (k[:-1] + 1), rtol=4 * n * EPS)
    assert np.array_equal(piv, np.arange(n))
    # partition closed form: {0}, {1}, ..., {n-3}, {n-2, n-1}
    exp = list(range(n - 1)) + [n] if n > 1 else [0, 1]
    assert list(o.sn_start) == exp
    # flops: each L(i, i-1) costs one division and one multiply-add
    assert o.flops[0] == 3 * (n - 1)


@pytest.mark.parametrize("seed", range(3))
def test_bidiagonal_solves_closed_form(seed):
    """B unit lower bidiagonal with B(i, i-1) = -a has the inverse
    B^-1(i, j) = a^(i-j) for j <= i.  A = P B Q^T (rows and columns permuted,
    values scaled by dr, dc inside the solver) is handed to the oracle with
    rowperm = p, colperm = q, so its Ahat is B itself up to the scalings:
    A x = b gives x[q[k]] = sum_{j<=k} a^(k-j) b[p[j]], and A^T z = g gives
    z[p[j]] = sum_{i>=j} a^(i-j) g[q[i]]."""
    rng = np.random.default_rng(600 + seed)
    n, a = 40, 0.5
    p = rng.permutation(n)
    q = rng.permutation(n)
    rows = np.concatenate([p, p[1:]])
    cols = np.concatenate([q, q[:-1]])
    vals = np.concatenate([np.ones(n), np.full(n - 1, -a)])
    A = synth.from_coo(n, rows, cols, vals)
    dr = rng.uniform(0.5, 2.0, n)
    dc = rng.uniform(0.5, 2.0, n)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, p, q, dr, dc)
    assert o.nperturb == 0
    b = rng.standard_normal(n)
    g = rng.standard_normal(n)
    x_cf = np.zeros(n)
    z_cf = np.zeros(n)
    for k in range(n):
        x_cf[q[k]] = sum(a ** (k - j) * b[p[j]] for j in range(k + 1))
        z_cf[p[k]] = sum(a ** (i - k) * g[q[i]] for i in range(k, n))
    np.testing.assert_allclose(o.solve(b), x_cf, rtol=0, atol=64 * EPS * np.abs(x_cf).max())
    np.testing.assert_allclose(o.solve_transpose(g), z_cf, rtol=0, atol=64 * EPS * np.abs(z_cf).max())


@pytest.mark.parametrize("n", [3, 10, 50])
def test_arrowhead_closed_form(n):
    """Diagonal d plus a dense last row r and last column c, natural order, no
    scaling.  U(k,:) = {k, n-1} for k < n-1, so L(n-1, k) = r_k / d_k costs one
    division and one multiply-add: 3 (n-1) flops.  Only the last two rows
    share a U structure: partition {0}, ..., {n-3}, {n-2, n-1}.  The last
    pivot is the Schur complement d_{n-1} - sum_k r_k c_k / d_k (with the
    supernode's pivoting: the larger of the last block's candidates)."""
    rng = np.random.default_rng(n)
    d = rng.uniform(4.0, 5.0, n)
    r = rng.uniform(-1, 1, n - 1)
    c = rng.uniform(-1, 1, n - 1)
    rows = list(range(n)) + [n - 1] * (n - 1) + list(range(n - 1))
    cols = list(range(n)) + list(range(n - 1)) + [n - 1] * (n - 1)
    A = synth.from_coo(n, rows, cols, list(d) + list(r) + list(c))
    o = oracle.Oracle(n, A.rowptr, A.col, A.val)
    assert o.flops[0] == 3 * (n - 1)
    assert list(o.sn_start) == list(range(n - 1)) + [n]
    L, U, piv = oracle.dense_factors(o)
    np.testing.assert_allclose(np.diag(U)[:n - 2], d[:n - 2], rtol=0, atol=0)
    # the last 2 x 2 block after eliminating rows 0..n-3, pivoted inside the supernode
    s = d[n - 1] - np.sum(r[:n - 2] * c[:n - 2] / d[:n - 2])
    blk = np.array([[d[n - 2], c[n - 2]], [r[n - 2], s]])
    a = np.zeros((n, n))
    a[np.arange(n), np.arange(n)] = d
    a[n - 1, :n - 1] = r
    a[:n - 1, n - 1] = c
    np.testing.assert_allclose(L @ U, a[:, piv], rtol=0, atol=1e-13)
    assert abs(np.prod(np.diag(U)[n - 2:])) == pytest.approx(abs(np.linalg.det(blk)), rel=1e-12)


def test_laplacian1d_scaled_pivots():
    """With diagonal scalings the pivots become dr_k * dc_k * (k+1)/k."""
    n = 20
    rng = np.random.default_rng(3)
    A = tridiag(n)
    dr = rng.uniform(0.5, 2, n)
    dc = rng.uniform(0.5, 2, n)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, dr=dr, dc=dc)
    _, _, ud = o.factors()
    k = np.arange(1, n + 1)
    np.testing.assert_allclose(ud, dr * dc * (k + 1) / k, rtol=8 * n * EPS)


def test_golden_dense2x2():
    g = read_golden("dense2x2_pivot.txt")
    a = g["A"].reshape(2, 2)
    A = dense_csr(a)
    o = oracle.Oracle(2, A.rowptr, A.col, A.val)
    L, U, piv = oracle.dense_factors(o)
    assert list(piv) == list(g["piv"].astype(int))
    np.testing.assert_array_equal(L, g["L"].reshape(2, 2))
    np.testing.assert_array_equal(U, g["U"].reshape(2, 2))


def test_golden_standalone_zero_pivot_and_refinement():
    g = read_golden("standalone_zero_pivot.txt")
    a = g["A"].reshape(3, 3)
    A = dense_csr(a + 0.0)
    # keep the explicit zero diagonal entries in the pattern
    A = synth.from_coo(3, [0, 0, 1, 2, 2], [0, 2, 1, 0, 2], [0.0, 1.0, 1.0, 1.0, 1.0])
    o = oracle.Oracle(3, A.rowptr, A.col, A.val)
    assert list(o.sn_start) == [0, 1, 2, 3]
    assert o.nperturb == int(g["nperturb"][0])
    _, _, ud = o.factors()
    assert ud[0] == o.tau == oracle.TAU_REL
    b = np.array([1.0, 2.0, 3.0])
    x, it, be = o.solve_refine(b)
    assert it >= 1 and be <= 1e-12
    np.testing.assert_allclose(x, g["Ainv"].reshape(3, 3) @ b, atol=1e-12)


def test_perturbation_sign():
    for v, sgn in ((1e-20, 1.0), (-1e-20, -1.0), (0.0, 1.0)):
        A = synth.from_coo(2, [0, 1], [0, 1], [v, 1.0])
        o = oracle.Oracle(2, A.rowptr, A.col, A.val)
        _, _, ud = o.factors()
        assert o.nperturb == 1 and ud[0] == sgn * o.tau


# -------------------------------------------- dense block vs LAPACK getrf
@pytest.mark.parametrize("n,seed", [(3, 0), (8, 1), (33, 2), (100, 3)])
def test_dense_supernode_matches_lapack_on_transpose(n, seed):
    """One dense supernode: row-wise largest-entry pivoting of Ahat equals
    LAPACK's partial pivoting (first max) of Ahat^T, rescaled to Doolittle."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    A = dense_csr(a)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, sn_max=256)
    assert list(o.sn_start) == [0, n]
    L, U, piv = oracle.dense_factors(o)
    P, Lt, Ut = sla.lu(a.T)            # a.T = P @ Lt @ Ut
    perm = np.argmax(P, axis=0)        # row perm[p] of a.T is at position p
    assert np.array_equal(piv, perm)
    d = np.diag(Ut)
    np.testing.assert_allclose(L, (Ut.T / d), atol=1e-12 * n)
    np.testing.assert_allclose(U, (d[:, None] * Lt.T), atol=1e-12 * n * np.abs(a).max())


def test_dense_split_by_sn_max():
    n = 40
    a = np.random.default_rng(5).standard_normal((n, n))
    A = dense_csr(a)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, sn_max=16)
    assert list(o.sn_start) == [0, 16, 32, 40]
    L, U, piv = oracle.dense_factors(o)
    assert np.linalg.norm(L @ U - a[:, piv]) <= 10 * n * EPS * np.linalg.norm(a) * 10


def test_block_diagonal_supernodes():
    rng = np.random.default_rng(7)
    sizes = [3, 1, 5, 2, 4]
    n = sum(sizes)
    a = np.zeros((n, n))
    s = 0
    for b in sizes:
        a[s:s + b, s:s + b] = rng.standard_normal((b, b)) + 3 * np.eye(b)
        s += b
    A = dense_csr(a)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val)
    assert list(o.sn_start) == list(np.concatenate([[0], np.cumsum(sizes)]))


def test_dense_flop_count():
    for n in (1, 2, 7, 30):
        a = np.random.default_rng(n).standard_normal((n, n)) + n * np.eye(n)
        A = dense_csr(a)
        o = oracle.Oracle(n, A.rowptr, A.col, A.val)
        assert o.flops[0] == n * (n - 1) / 2 + (n - 1) * n * (2 * n - 1) / 3


# ------------------------------------------ symbolic vs boolean elimination
def boolean_elimination(pat):
    """Dense boolean Gaussian elimination without cancellation."""
    B = pat.copy()
    n = B.shape[0]
    np.fill_diagonal(B, True)
    for k in range(n):
        rows = np.nonzero(B[k + 1:, k])[0] + k + 1
        B[np.ix_(rows, np.arange(k + 1, n))] |= B[k, k + 1:]
    return B


@pytest.mark.parametrize("seed", range(60))
def test_symbolic_matches_boolean_elimination(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 41))
    pat = rng.random((n, n)) < rng.uniform(0.02, 0.25)
    np.fill_diagonal(pat, True)
    a = np.where(pat, rng.uniform(-1, 1, (n, n)), 0.0)
    r, c = np.nonzero(pat)
    A = synth.from_coo(n, r, c, a[r, c])
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, numeric=False)
    F = o.unpadded
    got = np.zeros((n, n), bool)
    for i in range(n):
        got[i, F.col[F.rowptr[i]:F.rowptr[i + 1]]] = True
        assert np.all(np.diff(F.col[F.rowptr[i]:F.rowptr[i + 1]]) > 0)
    assert np.array_equal(got, boolean_elimination(pat))


# ------------------------------------------------- padded pattern invariants
def _rows(P, i):
    return P.col[P.rowptr[i]:P.rowptr[i + 1]]


@pytest.mark.parametrize("seed", range(20))
def test_padding_invariants(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(5, 60))
    a = random_sparse(n, rng.uniform(0.03, 0.2), rng)
    A = dense_csr(a)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, sn_max=int(rng.integers(2, 9)))
    F, P, sn = o.unpadded, o.padded, o.sn_start
    sn_of = np.repeat(np.arange(len(sn) - 1), np.diff(sn))
    for s in range(len(sn) - 1):
        r, e = sn[s], sn[s + 1] - 1
        first = _rows(P, r)
        for i in range(r, e + 1):
            f, p = _rows(F, i), _rows(P, i)
            assert set(f) <= set(p)
            assert np.array_equal(f[f >= i], p[p >= i][np.isin(p[p >= i], f)])
            # U structure unchanged outside the own block; block dense (rule i)
            assert np.array_equal(p[p > e], f[f > e])
            assert set(range(r, e + 1)) <= set(p)
            # every row of a supernode holds the same block and U tail
            assert np.array_equal(p[p >= r], first[first >= r])
            # rule ii: full supernode segments
            for k in p[p < r]:
                S = sn_of[k]
                assert set(range(sn[S], sn[S + 1])) <= set(p)
            # closure: every source's U(k, >k) lies in the row
            for k in p[p < i]:
                uk = _rows(P, k)
                assert set(uk[uk > k]) <= set(p)
            # exact L content: the row's own unpadded L columns before its
            # block, each widened to its source node's full segment, and
            # nothing more (no union over the rows of the supernode)
            want = set()
            for k in f[f < r]:
                S = sn_of[k]
                want |= set(range(sn[S], sn[S + 1]))
            assert np.array_equal(p[p < r], np.array(sorted(want), dtype=p.dtype))


def _golden_rows(name):
    g = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        g[k] = np.array([int(t) for t in v], dtype=np.int64)
    return g


def test_golden_padded_pattern():
    # tests/golden/padded_pattern_6.txt: a source supernode {0,1} feeding a
    # standalone row (2) and a supernode row (3), and a supernode {3,4} whose
    # second row keeps its own L column only
    g = _golden_rows("padded_pattern_6.txt")
    n = 6
    a = np.zeros((n, n))
    rng = np.random.default_rng(5)
    for i in range(n):
        a[i, g[f"A{i}"]] = rng.uniform(1.0, 2.0, len(g[f"A{i}"]))
    a += 10.0 * np.eye(n)
    A = dense_csr(a)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, sn_max=8)
    F, P = o.unpadded, o.padded
    assert np.array_equal(o.sn_start, g["sn"])
    for i in range(n):
        assert np.array_equal(_rows(F, i), g[f"F{i}"]), i
        assert np.array_equal(_rows(P, i), g[f"P{i}"]), i


# -------------------------------------------- reconstruction and solves
@pytest.mark.parametrize("seed", range(12))
def test_reconstruction_and_solve(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 120))
    a = random_sparse(n, rng.uniform(0.02, 0.15), rng, dominant=bool(seed % 2))
    A = dense_csr(a)
    rowperm = rng.permutation(n)
    colperm = rng.permutation(n)
    dr = rng.uniform(0.5, 2, n)
    dc = rng.uniform(0.5, 2, n)
    o = oracle.Oracle(n, A.rowptr, A.col, A.val, rowperm, colperm, dr, dc, sn_max=8)
    ahat = (dr[:, None] * a * dc[None, :])[np.ix_(rowperm, colperm)]
    L, U, piv = oracle.dense_factors(o)
    assert np.allclose(np.tril(L), L) and np.allclose(np.triu(U), U)
    # a perturbed pivot makes L U the factorization of Ahat Pi + diag(delta),
    # |delta_k| <= tau, nonzero only at the perturbed positions (Sec. 2.2)
    # componentwise backward error bound of LU (Higham, Thm. 9.3):
    # |L U - Ahat Pi| <= gamma_n |L| |U|, gamma_n = n eps / (1 - n eps)
    D = L @ U - ahat[:, piv]
    bound = 2 * n * EPS * (np.abs(L) @ np.abs(U)) + 1e-300
    off = ~np.eye(n, dtype=bool)
    assert np.all(np.abs(D[off]) <= bound[off])
    big = np.abs(np.diag(D)) > np.diag(bound)
    assert big.sum() <= o.nperturb
    assert np.all(np.abs(np.diag(D)) <= o.tau + np.diag(bound))
    if o.nperturb == 0:
        assert np.linalg.norm(D) <= 10 * n * EPS * np.linalg.norm(np.abs(L) @ np.abs(U))
    b = rng.standard_normal(n)
    xt = np.linalg.solve(a, b)
    yt = np.linalg.solve(a.T, b)
    cond = np.linalg.cond(a)
    if o.nperturb == 0:
        x = o.solve(b)
        assert np.abs(x - xt).max() <= 1e3 * cond * EPS * max(1, np.abs(xt).max())
        y = o.solve_transpose(b)
        assert np.abs(y - yt).max() <= 1e3 * cond * EPS * max(1, np.abs(yt).max())
    x2, _, be = o.solve_refine(b, force=True)
    if cond < 1e6 and o.nperturb == 0:
        assert be <= 1e-12


def test_workload_small_cases_backward_error():
    for m in (synth.grid5(16), synth.circuit(3000, seed=11), synth.convdiff3d(8),
              synth.aniso9(24)):
        o = oracle.Oracle(m.n, m.rowptr, m.col, m.val)
        xt, b = synth.rhs(m, 1)
        x, _, be = o.solve_refine(b[0], force=True)
        assert be <= 1e-12, be


# ------------------------------------------------- backward error (Sec. 2.3)
def _dense_backward_error(a, x, b):
    # ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), ||A||_inf the
    # largest absolute row sum
    r = b - a @ x
    return np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max())


def test_backward_error_hand_case():
    # row sums 3, 0.5, 0.5 (||A||_inf = 3) but column sums 1, 1.5, 1.5
    # (||A||_1 = 1.5): x = (1, 2, 3), b = (1, 1, 1) -> A x = (6, 1, 1.5),
    # r = (-5, 0, -0.5), so the error is 5 / (3 * 3 + 1) = 0.5 exactly.  The
    # column-sum norm would give 5 / 5.5, the 1-norms 5.5 / 12, and a dropped
    # ||b|| term 5 / 9.
    a = np.array([[1.0, 1.0, 1.0], [0.0, 0.5, 0.0], [0.0, 0.0, 0.5]])
    A = dense_csr(a)
    x = np.array([1.0, 2.0, 3.0])
    b = np.ones(3)
    assert oracle.backward_error(3, A.rowptr, A.col, A.val, x, b) == 0.5


def test_backward_error_zero_denominator():
    # x = 0 and b = 0: the residual is 0 and so is the error
    A = dense_csr(np.array([[2.0, 1.0], [0.0, 3.0]]))
    assert oracle.backward_error(2, A.rowptr, A.col, A.val, np.zeros(2), np.zeros(2)) == 0.0


@pytest.mark.parametrize("seed", range(8))
def test_backward_error_matches_dense(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(3, 80))
    a = random_sparse(n, rng.uniform(0.05, 0.3), rng)
    a[rng.integers(n), :] *= 7.0          # one heavy row: row and column norms differ
    A = dense_csr(a)
    x = rng.standard_normal(n) * rng.uniform(0.1, 10.0)
    b = rng.standard_normal(n)
    got = oracle.backward_error(n, A.rowptr, A.col, A.val, x, b)
    want = _dense_backward_error(a, x, b)
    assert abs(got - want) <= 1e-13 * want
    # the exact solution of a diagonally dominant system has an error near eps
    a2 = a + np.diag(np.abs(a).sum(axis=1) + 1.0)
    A2 = dense_csr(a2)
    xs = np.linalg.solve(a2, b)
    assert oracle.backward_error(n, A2.rowptr, A2.col, A2.val, xs, b) <= 1e-15 * n
