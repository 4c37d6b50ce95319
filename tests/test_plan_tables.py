"""Tables of the plan that the factor kernel reads without checking, verified
on the host from the plan image (hylu_plan_save):

- the value scatter (Sec. 2.1 scaling and permutation, then the row storage of
  Sec. 2.2): entry t of Ahat row i takes A's value at ah_src[t] (an entry of
  original row rowperm[i]), times ah_scale[t] = dr[rowperm[i]] dc[col], and
  lands in the slot of its permuted column in row i's storage -- its L list,
  its supernode's diagonal block, or the node's U tail;
- the tail tasks: the 32-column groups of a supernode's U tail are split over
  node_ntask[D] tasks, task t taking groups task_chunk[t], + node_ntask, ...;
  every group is solved by exactly one task;
- the panel offsets: node D's dense panel holds s x (s + |tail|) values."""
import numpy as np
import pytest

from paper_2509_07690_gb300 import Solver, synth
from plan_image import PlanImage

CASES = [
    ("grid5_20", lambda: synth.grid5(20), {}),
    ("circuit_3000", lambda: synth.circuit(3000, seed=14), {}),
    ("convdiff_10_nd", lambda: synth.convdiff3d(10), {"ordering": 1}),
    ("aniso_24_nd_sn9", lambda: synth.aniso9(24), {"ordering": 1, "sn_max": 9}),
    ("circuit_800_natural", lambda: synth.circuit(800, seed=2), {"ordering": 2}),
    ("circuit_3000_nd", lambda: synth.circuit(3000, seed=12), {"ordering": 1}),
]


def check_scatter(img):
    n = img.n
    qinv = np.empty(n, np.int64)
    qinv[img.colperm] = np.arange(n)
    sn, node_of = img.sn_start, img.node_of
    for i in range(n):
        D = node_of[i]
        r, e = sn[D], sn[D + 1] - 1
        s = e - r + 1
        lc = img.lcols[img.row_lptr[i]:img.row_lptr[i + 1]]
        tc = img.tcols[img.node_tail_off[D]:img.node_tail_off[D + 1]]
        nL = len(lc)
        t0, t1 = img.ah_rp[i], img.ah_rp[i + 1]
        src = img.ah_src[t0:t1]
        orow = img.rowperm[i]
        # the entries of original row rowperm[i], each once
        assert np.array_equal(np.sort(src), np.arange(img.a_rp[orow], img.a_rp[orow + 1]))
        ocol = img.a_ci[src]
        k = qinv[ocol]
        assert np.all(np.diff(k) > 0)                           # sorted by permuted column
        assert np.array_equal(img.ah_scale[t0:t1], img.dr[orow] * img.dc[ocol])
        slot = img.ah_slot[t0:t1]
        for kk, sl in zip(k, slot):
            if kk < r:
                assert sl < nL and lc[sl] == kk
            elif kk <= e:
                assert sl == nL + (kk - r)
            else:
                assert nL + s <= sl < nL + s + len(tc) and tc[sl - nL - s] == kk


def check_tasks(img):
    sn = img.sn_start
    for D in range(img.nnodes):
        s = sn[D + 1] - sn[D]
        nT = img.node_tail_off[D + 1] - img.node_tail_off[D]
        assert img.node_panel_off[D + 1] - img.node_panel_off[D] == s * (s + nT)
        m = img.node_ntask[D]
        tasks = np.nonzero(img.task_node == D)[0]
        if s < 2 or nT == 0:
            assert m == 0 and len(tasks) == 0
            continue
        ngroups = (nT + 31) // 32
        assert len(tasks) == m and m <= ngroups
        if m:
            assert sorted(img.task_chunk[tasks].tolist()) == list(range(m))
            covered = sorted(g for t in tasks for g in range(img.task_chunk[t], ngroups, m))
            assert covered == list(range(ngroups))
            # a tail task sits one level after its node's last row
            assert np.all(img.task_level[tasks] == img.row_level[sn[D + 1] - 1] + 1)
    check_claim_order(img)


def check_claim_order(img):
    """The factor kernel's main queue is a topological order of its
    dependencies: a supernode's rows in index order, its tail tasks after its
    last row, and a row after every row and tail task of each node its L list
    reads (progress of the persistent kernel rests on that)."""
    n, sn = img.n, img.sn_start
    order = img.row_order
    assert sorted(order.tolist()) == list(range(n + len(img.task_node)))
    at = np.empty(len(order), np.int64)
    at[order] = np.arange(len(order))
    done = np.empty(img.nnodes, np.int64)      # position of the node's last claim
    for D in range(img.nnodes):
        rows = np.arange(sn[D], sn[D + 1])
        assert np.all(np.diff(at[rows]) > 0)
        done[D] = at[rows[-1]]
        tasks = np.nonzero(img.task_node == D)[0]
        if len(tasks):
            assert np.all(at[n + tasks] > at[rows[-1]])
            done[D] = at[n + tasks].max()
    node_of = img.node_of
    for i in range(n):
        lc = img.lcols[img.row_lptr[i]:img.row_lptr[i + 1]]
        if len(lc):
            assert at[i] > done[np.unique(node_of[lc])].max(), i


@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_scatter_map_and_tail_tasks(name, make, opts):
    A = make()
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    img = PlanImage(s.save())
    s.close()
    assert np.array_equal(img.a_rp, A.rowptr) and np.array_equal(img.a_ci, A.col)
    check_scatter(img)
    check_tasks(img)


def test_scatter_map_of_a_batch():
    """In a batch the same relations hold on the combined system; ah_src
    indexes the concatenated values (instance q from val_base[q])."""
    from paper_2509_07690_gb300 import BatchSolver
    mats = [synth.circuit(500, seed=3), synth.grid5(9), synth.aniso9(10)]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], 3)
    img = PlanImage(bs.save())
    bs.close()
    for q in range(9):
        v, sidx = divmod(q, 3)
        m = mats[sidx]
        rb, vb = img.row_base[q], img.val_base[q]
        assert np.array_equal(img.a_rp[rb:rb + m.n + 1] - img.a_rp[rb], m.rowptr)
        assert img.a_rp[rb] == vb
        assert np.array_equal(img.a_ci[vb:vb + m.nnz] - rb, m.col)
    check_scatter(img)
    check_tasks(img)


def test_checks_detect_planted_mistakes():
    """Mistakes planted in copies of the tables, not in the library."""
    A = synth.convdiff3d(8)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1)
    image = s.save()
    s.close()
    img = PlanImage(image)
    t = int(np.nonzero(np.diff(img.ah_rp))[0][5])
    img.ah_slot = img.ah_slot.copy()
    img.ah_slot[img.ah_rp[t]] += 1
    with pytest.raises(AssertionError):
        check_scatter(img)
    img = PlanImage(image)
    img.ah_scale = img.ah_scale.copy()
    img.ah_scale[7] *= 1.0 + 2.0 ** -40
    with pytest.raises(AssertionError):
        check_scatter(img)
    img = PlanImage(image)
    assert np.any(img.node_ntask > 1)                  # a node split over several tail tasks
    D = int(np.nonzero(img.node_ntask > 1)[0][0])
    tasks = np.nonzero(img.task_node == D)[0]
    img.task_chunk = img.task_chunk.copy()
    img.task_chunk[tasks[0]] = img.task_chunk[tasks[1]]
    with pytest.raises(AssertionError):
        check_tasks(img)
