"""The seeded generators follow the configurations' recipes: sizes and entry
counts, structure (stencils, band, hubs), value distributions and the
properties the discretisations imply."""
import numpy as np

from paper_2509_07690_gb300 import synth


def _rows(m):
    return np.repeat(np.arange(m.n), np.diff(m.rowptr))


def _transpose_values(m):
    """Values of A^T on A's pattern (the pattern must be symmetric)."""
    rid = _rows(m)
    key = rid.astype(np.int64) * m.n + m.col
    tkey = m.col.astype(np.int64) * m.n + rid
    order = np.argsort(key)
    pos = np.searchsorted(key[order], tkey)
    assert np.array_equal(key[order][pos], tkey), "pattern not symmetric"
    return m.val[order][pos]


def test_grid5_64():
    m = synth.workload("grid5_64")
    assert m.n == 4096 and m.nnz == 20224
    rid = _rows(m)
    d = m.col == rid
    assert np.all((m.val[d] >= 4.0) & (m.val[d] < 4.1))
    assert np.all((m.val[~d] >= -1.2) & (m.val[~d] <= -0.8))
    off = np.abs(m.col[~d] - rid[~d])
    assert set(np.unique(off)) == {1, 64}
    assert np.all(np.diff(m.rowptr) <= 5)
    assert not np.allclose(m.val, _transpose_values(m))       # unsymmetric values


def test_circuit_100k():
    m = synth.workload("circuit_100k")
    assert m.n == 100_000 and 1.3e6 <= m.nnz <= 1.5e6
    rid = _rows(m)
    cnt = np.diff(m.rowptr)
    hub_rows = np.nonzero(cnt > 100)[0]
    assert len(hub_rows) == 1000                              # 1% of the indices
    assert cnt[hub_rows].min() >= 150 and cnt[hub_rows].max() <= 2000 + 100
    # hub columns: the columns with more than 100 entries
    colcnt = np.bincount(m.col, minlength=m.n)
    hub_cols = set(np.nonzero(colcnt > 100)[0].tolist())
    assert len(hub_cols) == 1000
    # a non-hub row's off-diagonals lie in the +-50 band or in a hub column
    d = m.col == rid
    nonhub = ~np.isin(rid, hub_rows) & ~d
    far = np.abs(m.col[nonhub] - rid[nonhub]) > 50
    assert all(c in hub_cols for c in np.unique(m.col[nonhub][far]).tolist())
    # values: off-diagonals U(-1, 1); diagonal = +-rowabs x U(1, 1.5)
    assert np.all(np.abs(m.val[~d]) <= 1.0)
    rowabs = np.bincount(rid[~d], weights=np.abs(m.val[~d]), minlength=m.n)
    ratio = np.abs(m.val[d]) / rowabs[rid[d]]
    assert ratio.min() >= 1.0 - 1e-12 and ratio.max() <= 1.5 + 1e-12
    assert 0.4 < np.mean(m.val[d] > 0) < 0.6                  # random signs


def test_convdiff3d_64():
    m = synth.workload("convdiff3d_64")
    assert m.n == 64 ** 3 and m.nnz == 1_810_432
    rid = _rows(m)
    cnt = np.diff(m.rowptr)
    assert cnt.max() == 7
    # upwind: zero row sums inside the grid (an M-matrix), positive on the boundary
    rs = np.bincount(rid, weights=m.val, minlength=m.n)
    assert np.all(np.abs(rs[cnt == 7]) < 1e-12)
    assert np.all(rs[cnt < 7] > 0)
    d = m.col == rid
    assert np.all(m.val[~d] < 0)
    # cell Peclet 10 along (1, 0.5, 0.25): the strongest coupling is 1 + |v_x|
    v = 2.0 * 10.0 * np.array([1.0, 0.5, 0.25]) / np.linalg.norm([1.0, 0.5, 0.25])
    assert np.isclose(-m.val[~d].min(), 1.0 + v[0])
    assert not np.allclose(m.val, _transpose_values(m))       # convection: unsymmetric


def test_aniso9_512():
    m = synth.workload("aniso9_512")
    assert m.n == 512 ** 2 and m.nnz == 2_353_156
    assert np.diff(m.rowptr).max() == 9
    assert np.allclose(m.val, _transpose_values(m), rtol=0, atol=1e-12)   # -div(K grad) is symmetric
    rid = _rows(m)
    d = m.col == rid
    assert np.all(m.val[d] > 0)
    # log-normal coefficients: the diagonal spans orders of magnitude
    assert m.val[d].max() / m.val[d].min() > 10.0


def test_batch_sizes_and_determinism():
    s = synth.circuit_batch_sizes()
    assert len(s) == 512 and s.min() >= 2000 and s.max() <= 40000
    assert np.array_equal(s, synth.circuit_batch_sizes())
    a = synth.circuit(3000, seed=9)
    b = synth.circuit(3000, seed=9)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)
    c = synth.circuit_value_set(a, 5)
    assert np.array_equal(c.col, a.col) and not np.array_equal(c.val, a.val)
