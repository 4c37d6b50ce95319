"""Host partition of the bulk-sequential substitution (HYLU Sec. 2.3, Fig. 3:
levels with many nodes are solved in bulk, the long chain sequentially),
rebuilt here by brute force and compared entry by entry.

The brute force starts from the exported padded pattern: the forward level of
a node is one past the highest level of the nodes its rows' L entries lie in,
the backward level one past the highest level of the nodes its U tail columns
lie in.  A level is light when it holds at most max_rows rows, no node of more
rows, and at most 1024 max_rows entries of work (L lists, or U tails times
the node's rows, plus the squared node sizes); segments are the maximal
chains of two or more consecutive light levels of one instance."""
import numpy as np
import pytest

from paper_2509_07690_gb300 import BatchSolver, Solver, capi, synth
from plan_image import PlanImage


def _cases():
    rng = np.random.default_rng(5)
    a = rng.standard_normal((120, 120)) * (rng.random((120, 120)) < 0.05) + 8 * np.eye(120)
    r, c = np.nonzero(a)
    yield "random_120", synth.from_coo(120, r, c, a[r, c]), {}
    yield "circuit_3000", synth.circuit(3000, seed=2), {}
    yield "grid5_24_amd", synth.grid5(24), {}
    yield "convdiff_10_nd", synth.convdiff3d(10), {"ordering": 1}


CASES = list(_cases())


def _levels(s):
    """Forward and backward node levels, node sizes and per-node work, from
    the exported pattern alone."""
    n = s.n
    rp, ci = s.export_pattern()
    sn = s.export_perm()[4]
    nn = len(sn) - 1
    node_of = np.repeat(np.arange(nn), np.diff(sn))
    size = np.diff(sn)
    fl = np.zeros(nn, np.int64)
    lwork = np.zeros(nn, np.int64)
    for D in range(nn):
        for i in range(sn[D], sn[D + 1]):
            row = ci[rp[i]:rp[i + 1]]
            lc = row[row < sn[D]]
            lwork[D] += len(lc)
            if len(lc):
                fl[D] = max(fl[D], fl[node_of[lc]].max() + 1)
    bl = np.zeros(nn, np.int64)
    tails = []
    for D in reversed(range(nn)):
        row = ci[rp[sn[D]]:rp[sn[D] + 1]]
        tail = row[row >= sn[D + 1]]
        tails.append(len(tail))
        if len(tail):
            bl[D] = bl[node_of[tail]].max() + 1
    tails = np.array(tails[::-1], np.int64)
    fwork = lwork + size * size
    bwork = size * tails + size * size
    return dict(sn=sn, size=size, node_of=node_of, fl=fl, bl=bl, fwork=fwork, bwork=bwork)


def _brute_segments(level, size, work, inst, max_rows):
    """Segments as (instance, first level, last level), sorted by first level."""
    segs = []
    if max_rows <= 0:
        return segs
    for q in np.unique(inst):
        sel = inst == q
        L = int(level[sel].max()) + 1
        rows = np.bincount(level[sel], weights=size[sel], minlength=L)
        big = np.zeros(L, np.int64)
        np.maximum.at(big, level[sel], size[sel])
        wk = np.bincount(level[sel], weights=work[sel], minlength=L)
        light = (rows <= max_rows) & (big <= max_rows) & (wk <= 1024 * max_rows)
        l = 0
        while l < L:
            if not light[l]:
                l += 1
                continue
            e = l
            while e + 1 < L and light[e + 1]:
                e += 1
            if e > l:
                segs.append((l, int(q), e))
            l = e + 1
    return [(q, l0, l1) for (l0, q, l1) in sorted(segs)]


def _check(S, segs, level, inst, sn, order):
    assert S["meta"].tolist() == [list(g) for g in segs]
    assert len(S["seg_off"]) == len(segs) + 1
    in_seg = np.zeros(len(sn) - 1, bool)
    k = 0
    for g, (q, l0, l1) in enumerate(segs):
        assert S["seg_off"][g] == k and S["seg_off"][g + 1] == k + l1 - l0 + 1
        for l in range(l0, l1 + 1):
            nodes = np.nonzero((level == l) & (inst == q))[0]
            in_seg[nodes] = True
            want_rows = np.concatenate([np.arange(sn[D], sn[D + 1]) for D in nodes])
            got_rows = S["rows"][S["lvl_row"][k]:S["lvl_row"][k + 1]]
            assert np.array_equal(got_rows, want_rows)
            want_sn = [D for D in nodes if sn[D + 1] - sn[D] > 1]
            assert S["snodes"][S["lvl_node"][k]:S["lvl_node"][k + 1]].tolist() == want_sn
            k += 1
    assert len(S["lvl_row"]) == k + 1
    # the bulk claim list: the rows outside the segments, in their claim order
    # (entries from n on are the forward long rows' chunks)
    node_of = np.repeat(np.arange(len(sn) - 1), np.diff(sn))
    n = len(node_of)
    want_task = [i for i in order if not in_seg[node_of[i]]]
    rows_task = [int(t) for t in S["task"] if t < n]
    assert rows_task == want_task
    assert len(rows_task) + len(S["rows"]) == len(order)


def _check_chunks(S, level, node_of, lptr, lcols, backward):
    """Forward long rows (at least 2048 L entries, outside the segments): their
    lists in ceil(nL / 1024) chunks of near-equal length, each waiting for one
    past the highest level of its entries' sources and claimed before every
    row of that level or later (after every row of a lower level)."""
    n = len(node_of)
    task = S["task"]
    if backward:
        assert len(S["chunk_row"]) == 0 and np.all(S["row_chunk_off"] == 0)
        assert np.all(task < n)
        return
    want = []
    for i in task[task < n]:
        nl = lptr[i + 1] - lptr[i]
        if nl < 2048:
            continue
        nc = -(-nl // 1024)
        for c in range(nc):
            a, b = c * nl // nc, (c + 1) * nl // nc
            src = lcols[lptr[i] + a:lptr[i] + b]
            want.append((int(i), int(a), int(b), int(level[node_of[src]].max() + 1)))
    got = list(zip(S["chunk_row"].tolist(), S["chunk_a"].tolist(), S["chunk_b"].tolist(), S["chunk_level"].tolist()))
    assert sorted(got) == sorted(want)
    cnt = np.bincount(S["chunk_row"], minlength=n) if len(got) else np.zeros(n, np.int64)
    assert np.array_equal(np.diff(S["row_chunk_off"]), cnt)
    for c, (i, a, b, lv) in enumerate(got):
        assert S["row_chunk_off"][i] <= c < S["row_chunk_off"][i + 1]
    # placement: the highest level of the rows before each chunk entry is below
    # the chunk's level, the lowest level of the rows after it is not
    is_row = task < n
    lv_rows = np.where(is_row, level[node_of[np.where(is_row, task, 0)]], 0).astype(np.int64)
    before = np.maximum.accumulate(np.where(is_row, lv_rows, -1))
    after = np.minimum.accumulate(np.where(is_row, lv_rows, np.iinfo(np.int64).max)[::-1])[::-1]
    for k in np.nonzero(~is_row)[0]:
        lv = S["chunk_level"][task[k] - n]
        assert k == 0 or before[k - 1] < lv
        assert k == len(task) - 1 or after[k + 1] >= lv


@pytest.mark.parametrize("max_rows", [0, 1, 4, 16, 64])
@pytest.mark.parametrize("name,A,opts", CASES, ids=[c[0] for c in CASES])
def test_segments_match_brute_force(name, A, opts, max_rows):
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    B = _levels(s)
    img = PlanImage(capi.hylu_plan_save(s.h))
    # the plan's own levels are the brute-force ones
    assert np.array_equal(img.fwd_level, B["fl"])
    assert np.array_equal(img.bwd_level, B["bl"])
    inst = np.zeros(len(B["size"]), np.int64)
    for bwd, level, work, order in ((0, B["fl"], B["fwork"], img.fwd_order), (1, B["bl"], B["bwork"], img.bwd_order)):
        S = capi.hylu_export_solve_segments(s.h, bwd, max_rows)
        segs = _brute_segments(level, B["size"], work, inst, max_rows)
        _check(S, segs, level, inst, B["sn"], order)
        _check_chunks(S, level, B["node_of"], img.row_lptr, img.lcols, bwd)
    s.close()


@pytest.mark.parametrize("name,A,opts", [("circuit_12000", synth.circuit(12000, seed=9), {}),
                                         ("convdiff_40_nd", synth.convdiff3d(40), {"ordering": 1})],
                         ids=["circuit_12000", "convdiff_40_nd"])
def test_long_rows_split_into_chunks(name, A, opts):
    """Matrices whose long rows have more than 2048 L entries (circuit hub
    rows; a 3D grid's separators, whose claim order is not their index order):
    the forward partition splits them (the test above would pass without any),
    and every row's chunk range names its own chunks."""
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    img = PlanImage(capi.hylu_plan_save(s.h))
    S = capi.hylu_export_solve_segments(s.h, 0, 8)
    assert len(S["chunk_row"]) > 100
    node_of = np.repeat(np.arange(len(img.sn_start) - 1), np.diff(img.sn_start))
    _check_chunks(S, img.fwd_level, node_of, img.row_lptr, img.lcols, False)
    s.close()


def test_segments_found_on_a_chain():
    """The circuit matrix's forward solve ends in a long chain of small levels:
    the partition must put most of them in segments (else the test above may
    pass on empty partitions)."""
    A = synth.circuit(3000, seed=2)
    s = Solver(A.n, A.rowptr, A.col, A.val)
    S = capi.hylu_export_solve_segments(s.h, 0, 16)
    assert len(S["meta"]) >= 1 and len(S["lvl_row"]) - 1 >= 8
    s.close()


def test_batch_segments_per_instance():
    """A batch: levels and light levels are per instance; segments of all
    instances sorted by first level (then instance)."""
    mats = [synth.circuit(n, seed=q) for q, n in enumerate((900, 1400, 700))]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], nsets=2)
    img = PlanImage(capi.hylu_plan_save(bs.h))
    sn = img.sn_start
    size = np.diff(sn).astype(np.int64)
    inst = img.node_instance().astype(np.int64)
    lw = np.diff(img.row_lptr)
    node_of = np.repeat(np.arange(len(size)), size)
    lwork = np.bincount(node_of, weights=lw, minlength=len(size)).astype(np.int64)
    tails = np.diff(img.node_tail_off).astype(np.int64)
    for bwd, level, work, order in ((0, img.fwd_level, lwork + size * size, img.fwd_order),
                                    (1, img.bwd_level, size * tails + size * size, img.bwd_order)):
        S = capi.hylu_export_solve_segments(bs.h, bwd, 16)
        segs = _brute_segments(level.astype(np.int64), size, work, inst, 16)
        assert len(segs) > 0 or bwd == 1
        _check(S, segs, level, inst, sn, order)
        _check_chunks(S, level, node_of, img.row_lptr, img.lcols, bwd)
    bs.close()


def test_export_length_protocol():
    """hylu_export_solve_segments: a NULL buffer returns the length; a buffer
    too short is refused with HYLU_ERR_ARG and the length needed."""
    import ctypes as C
    A = synth.circuit(3000, seed=2)
    s = Solver(A.n, A.rowptr, A.col, A.val)
    lib = capi.load()
    need = C.c_int64(0)
    assert lib.hylu_export_solve_segments(s.h, 0, 8, None, C.byref(need)) == 0
    assert need.value > A.n
    short = C.c_int64(need.value - 1)
    buf = np.zeros(need.value, np.int32)
    assert lib.hylu_export_solve_segments(s.h, 0, 8, buf.ctypes.data, C.byref(short)) == -1
    assert short.value == need.value
    full = capi.hylu_export_solve_segments(s.h, 0, 8)
    assert len(full["row_chunk_off"]) == A.n + 1
    s.close()
