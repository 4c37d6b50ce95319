"""The substitution kernels' schedules, checked on the host from the plan
image (hylu_plan_save): forward L, backward U, and the transpose passes U^T
and L^T (Sec. 2.3, bulk mode of Sec. 2.2.1).

Each kernel claims rows in its order; a row of level L waits until its
instance's watermark reaches L (every level below complete); inside a
supernode, rows wait on the owner of their 32-row tile or on earlier tiles.
The checks:

- every data dependency of a node (L sources forward, U tail columns
  backward, the pushes of the transpose passes) lies at a strictly lower
  level of the same instance, so the watermark orders every read after its
  write;
- the level counts are each instance's node (L, U) or row (U^T, L^T) counts,
  with no empty level (an empty level would never complete);
- one warp that takes the rows in claim order finds every wait already
  satisfied: each row waits only on rows claimed before it, so no number of
  warps can deadlock.  The simulation follows the kernels' rules: forward,
  the last row of a tile owns it and the last tile completes the node;
  backward, the first row of a tile owns it and the first tile completes the
  node; U^T, the first row of a tile solves it and every row completes
  itself; L^T, the last row of a tile solves it, later tiles first."""
import numpy as np
import pytest

from paper_2509_07690_gb300 import Solver, synth
from plan_image import PlanImage


def _dense(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 1, (n, n)) + n * np.eye(n)
    r, c = np.nonzero(a)
    return synth.from_coo(n, r, c, a[r, c])


CASES = [
    ("grid5_16", lambda: synth.grid5(16), {}),
    ("circuit_3000", lambda: synth.circuit(3000, seed=12), {}),
    ("convdiff_10_nd", lambda: synth.convdiff3d(10), {"ordering": 1}),
    ("aniso_24_nd", lambda: synth.aniso9(24), {"ordering": 1}),
    ("convdiff_8_sn7", lambda: synth.convdiff3d(8), {"ordering": 1, "sn_max": 7}),
    ("dense_100", lambda: _dense(100, 3), {}),
    ("circuit_3000_nd", lambda: synth.circuit(3000, seed=12), {"ordering": 1}),
]


def _image(make, opts):
    A = make()
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    img = PlanImage(s.save())
    s.close()
    return img


def _batch_image():
    from paper_2509_07690_gb300 import BatchSolver
    mats = [synth.circuit(400, seed=8), synth.grid5(7), _dense(70, 4), synth.convdiff3d(6)]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], 2)
    img = PlanImage(bs.save())
    bs.close()
    return img


def _nodes(img):
    sn = img.sn_start
    return sn, img.node_of, np.diff(sn)


def check_dependencies(img):
    sn, node_of, size = _nodes(img)
    inst = img.node_instance()
    for D in range(img.nnodes):
        tail = img.tcols[img.node_tail_off[D]:img.node_tail_off[D + 1]]
        for T in np.unique(node_of[tail]):
            assert inst[T] == inst[D]
            assert img.bwd_level[T] < img.bwd_level[D]       # U w = z reads later nodes
            assert img.ut_level[D] < img.ut_level[T]         # U^T pushes into later nodes
        for i in range(sn[D], sn[D + 1]):
            lc = img.lcols[img.row_lptr[i]:img.row_lptr[i + 1]]
            for S in np.unique(node_of[lc]):
                assert inst[S] == inst[D]
                assert img.fwd_level[S] < img.fwd_level[D]   # L y = b reads earlier nodes
                assert img.lt_level[D] < img.lt_level[S]     # L^T pushes into earlier nodes


def check_counts(img, kind):
    sn, node_of, size = _nodes(img)
    inst = img.node_instance()
    level = getattr(img, kind + "_level")
    count = getattr(img, kind + "_count")
    off = img.slices(kind)
    per_row = kind in ("ut", "lt")
    ninst = len(off) - 1
    for q in range(ninst):
        nodes = np.nonzero(inst == q)[0]
        weights = size[nodes] if per_row else np.ones(len(nodes), np.int64)
        want = np.bincount(level[nodes], weights=weights).astype(np.int64)
        got = count[off[q]:off[q + 1]]
        assert np.array_equal(got, want), (kind, q)
        assert np.all(got >= 1), (kind, q, "empty level")


def simulate(img, kind):
    """One warp takes the rows in claim order; every wait must already hold."""
    sn, node_of, size = _nodes(img)
    inst = img.node_instance()
    order = getattr(img, kind + "_order")
    level = getattr(img, kind + "_level")
    count = getattr(img, kind + "_count")
    off = img.slices(kind)
    n = img.n
    assert np.array_equal(np.sort(order), np.arange(n))
    wm = np.zeros(len(off) - 1, np.int64)
    done = np.zeros(len(count), np.int64)
    pub = np.zeros(n, bool)        # per-row flags (fwd_row / bwd_row)
    tile = np.zeros(n, bool)       # tile flags, indexed as the kernels index them

    def complete(q, L):
        done[off[q] + L] += 1
        if done[off[q] + L] == count[off[q] + L]:
            wm[q] = L + 1

    for i in order:
        D = node_of[i]
        L, q = level[D], inst[D]
        r, e = sn[D], sn[D + 1] - 1
        assert wm[q] >= L, (kind, i, "watermark not reached")
        T0 = r + ((i - r) & ~31)
        if kind == "fwd":
            if r == e:
                complete(q, L)
                continue
            pub[i] = True
            tlast = min(T0 + 31, e)
            if i != tlast:
                continue
            assert pub[T0:tlast].all() and all(tile[K0 + 31] for K0 in range(r, T0, 32)), (kind, i)
            tile[tlast] = True
            if tlast == e:
                complete(q, L)
        elif kind == "bwd":
            if r == e:
                complete(q, L)
                continue
            pub[i] = True
            if i != T0:
                continue
            tl = min(T0 + 31, e)
            assert pub[T0 + 1:tl + 1].all(), (kind, i)
            assert all(tile[K0] for K0 in range(r + ((e - r) & ~31), T0, -32)), (kind, i)
            tile[T0] = True
            if T0 == r:
                complete(q, L)
        elif kind == "ut":
            if r < e:
                if i == T0:
                    assert all(tile[K0] for K0 in range(r, T0, 32)), (kind, i)
                    tile[T0] = True
                else:
                    assert tile[T0], (kind, i)
            complete(q, L)
        else:  # lt
            if r < e:
                tl = min(T0 + 31, e)
                if i == tl:
                    assert all(tile[min(K0 + 31, e)] for K0 in range(r + ((e - r) & ~31), T0, -32)), (kind, i)
                    tile[tl] = True
                else:
                    assert tile[tl], (kind, i)
            complete(q, L)
    for q in range(len(off) - 1):
        assert wm[q] == off[q + 1] - off[q], (kind, q, "levels left incomplete")


KINDS = ["fwd", "bwd", "ut", "lt"]


@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_substitution_schedules(name, make, opts):
    img = _image(make, opts)
    check_dependencies(img)
    for kind in KINDS:
        check_counts(img, kind)
        simulate(img, kind)


def test_substitution_schedules_batch():
    """Four systems x two value sets: per-instance levels, count slices and
    watermarks."""
    img = _batch_image()
    assert img.batch == 1 and len(img.node_inst) == img.nnodes
    assert len(img.fwd_off) == 4 * 2 + 1
    check_dependencies(img)
    for kind in KINDS:
        check_counts(img, kind)
        simulate(img, kind)


def test_simulation_detects_a_wrong_order():
    """Planted mistakes in copies of the schedule, not in the library: the
    forward order reversed, and a forward level lowered below a source's."""
    img = _image(lambda: synth.grid5(12), {})
    img.fwd_order = img.fwd_order[::-1].copy()
    with pytest.raises(AssertionError):
        simulate(img, "fwd")
    img = _image(lambda: _dense(40, 5), {"ordering": 2})
    assert img.sn_start.tolist() == [0, 40]              # one supernode of two tiles
    img.bwd_order = np.concatenate([img.bwd_order[8:], img.bwd_order[:8]])
    with pytest.raises(AssertionError):
        simulate(img, "bwd")
    img = _image(lambda: synth.grid5(12), {})
    D = int(np.argmax(img.fwd_level))
    img.fwd_level = img.fwd_level.copy()
    img.fwd_level[D] = 0
    with pytest.raises(AssertionError):
        check_dependencies(img)
