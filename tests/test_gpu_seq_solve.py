"""GPU parity of the bulk-sequential substitution (HYLU Sec. 2.3, Fig. 3):
with segments of light levels solved by one thread block each (and the
other rows in bulk), every solution has backward error <= 1e-12, agrees with
the oracle's solve (same pivots; the factors agree within 1e-10, so the
solutions within 1e-9) and with the all-bulk solve on the same factors
(solve_seq_rows = 0) within 1e-12, for one and several right-hand sides,
FP64 and FP32 factors, a single system and a batch.  Every case checks first
that the partition really has segments."""
import numpy as np
import pytest

import oracle
from paper_2509_07690_gb300 import BatchSolver, Solver, capi, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _nseg(h, max_rows):
    return [len(capi.hylu_export_solve_segments(h, d, max_rows)["meta"]) for d in (0, 1)]


CASES = [("circuit_3000", lambda: synth.circuit(3000, seed=2), {}),
         ("circuit_12000", lambda: synth.circuit(12000, seed=9), {}),
         ("grid5_40", lambda: synth.grid5(40, seed=3), {}),
         ("convdiff_12_nd", lambda: synth.convdiff3d(12), {"ordering": 1})]


@pytest.mark.parametrize("max_rows", [4, 16, 64])
@pytest.mark.parametrize("nrhs", [1, 3, 9])
@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_segments_vs_oracle(name, make, opts, nrhs, max_rows):
    torch = _torch()
    if name == "convdiff_12_nd" and max_rows < 16:
        max_rows = 16        # the 3D grid's levels hold more rows: no light chain below 10
    A = make()
    s = Solver(A.n, A.rowptr, A.col, A.val, solve_seq_rows=max_rows, **opts)
    assert sum(_nseg(s.h, max_rows)) > 0, "no segment: the case does not test the sequential mode"
    s.factor(torch.from_numpy(A.val).cuda())
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc)
    _, opiv, _ = o.factors()
    _, gpiv = s.export_factors()
    assert np.array_equal(opiv, gpiv)
    _, b = synth.rhs(A, 11, nrhs)
    x = s.solve(torch.from_numpy(b).cuda()).cpu().numpy().reshape(nrhs, A.n)
    bulk = Solver(A.n, A.rowptr, A.col, A.val, solve_seq_rows=0, **opts)
    assert _nseg(bulk.h, 0) == [0, 0]
    bulk.factor(torch.from_numpy(A.val).cuda())
    xb = bulk.solve(torch.from_numpy(b).cuda()).cpu().numpy().reshape(nrhs, A.n)
    for r in range(nrhs):
        assert oracle.backward_error(A.n, A.rowptr, A.col, A.val, x[r], b[r]) <= 1e-12, r
        xo = o.solve(b[r])
        assert np.linalg.norm(x[r] - xo) <= 1e-9 * np.linalg.norm(xo), r
        assert np.linalg.norm(x[r] - xb[r]) <= 1e-12 * np.linalg.norm(xb[r]), r
    assert s.get_info().device_status == 0
    s.close()
    bulk.close()


def test_segments_fp32_factors():
    torch = _torch()
    A = synth.circuit(12000, seed=9)
    s = Solver(A.n, A.rowptr, A.col, A.val, precision=1, solve_seq_rows=32)
    assert sum(_nseg(s.h, 32)) > 0
    s.factor(torch.from_numpy(A.val).cuda())
    _, b = synth.rhs(A, 5, 2)
    x = s.solve(torch.from_numpy(b).cuda()).cpu().numpy().reshape(2, A.n)
    for r in range(2):
        assert oracle.backward_error(A.n, A.rowptr, A.col, A.val, x[r], b[r]) <= 1e-12
    s.close()


def test_segments_transpose_unchanged():
    """The transpose solve has no sequential mode; it must still agree with
    the oracle on a plan that has segments."""
    torch = _torch()
    A = synth.circuit(3000, seed=2)
    s = Solver(A.n, A.rowptr, A.col, A.val, solve_seq_rows=16)
    s.factor(torch.from_numpy(A.val).cuda())
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc)
    _, g = synth.rhs(A, 12, 1)
    y = s.solve(torch.from_numpy(g[0]).cuda(), transpose=True).cpu().numpy()
    yo = o.solve_transpose(g[0])
    assert np.linalg.norm(y - yo) <= 1e-9 * np.linalg.norm(yo)
    s.close()


def test_segments_batch():
    """A batch: every instance's segments are claimed by the sequential blocks
    in order of first level; each instance's solution against the oracle run
    on that instance's own preprocessing outputs."""
    torch = _torch()
    mats = [synth.circuit(n, seed=20 + q) for q, n in enumerate((2500, 4000, 1800, 3200))]
    nsets = 2
    k = len(mats)
    value_sets = [[m.val if v == 0 else synth.circuit_values(m.rowptr, m.col, 70 + q) for q, m in enumerate(mats)]
                  for v in range(nsets)]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], nsets, solve_seq_rows=16)
    assert _nseg(bs.h, 16)[0] > 0
    bs.factor(torch.from_numpy(bs.concat_values(value_sets)).cuda())
    rp, cp, dr, dc, sn = bs.export_perm()
    b = np.random.default_rng(4).standard_normal((3, bs.n))
    x = bs.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    for v in range(nsets):
        for q, m in enumerate(mats):
            rb = bs.row_base[v * k + q]
            sl = slice(rb, rb + m.n)
            o = oracle.Oracle(m.n, m.rowptr, m.col, value_sets[v][q], rp[sl] - rb, cp[sl] - rb, dr[sl], dc[sl])
            for r in range(3):
                xo = o.solve(b[r, sl])
                assert oracle.backward_error(m.n, m.rowptr, m.col, value_sets[v][q], x[r, sl], b[r, sl]) <= 1e-12
                assert np.linalg.norm(x[r, sl] - xo) <= 1e-9 * np.linalg.norm(xo), (v, q, r)
    assert bs.get_info().device_status == 0
    bs.close()


def test_tuner_picks_a_segment_threshold():
    """hylu_tune times the substitution with the handle's solve_seq_rows and
    with every level in bulk, keeps the faster, and reports it; the solve is
    right either way."""
    torch = _torch()
    A = synth.circuit(12000, seed=9)
    s = Solver(A.n, A.rowptr, A.col, A.val, solve_seq_rows=16)
    dv = torch.from_numpy(A.val).cuda()
    s.factor(dv)
    info = s.get_info()
    assert info.solve_seq_rows == 16 and sum(info.solve_segments) > 0
    capi.hylu_tune(s.h, dv.data_ptr())
    info = s.get_info()
    assert info.tuned == 1 and info.solve_seq_rows in (16, 0)
    assert (sum(info.solve_segments) == 0) == (info.solve_seq_rows == 0)
    _, b = synth.rhs(A, 3, 1)
    x = s.solve(torch.from_numpy(b[0]).cuda()).cpu().numpy()
    assert oracle.backward_error(A.n, A.rowptr, A.col, A.val, x, b[0]) <= 1e-12
    s.close()


def test_many_segments_larger_launch_than_resident():
    """A batch with thousands of segments: the blocks that take the segments
    are the first to start, so their number is capped by what can be resident
    at once (a quarter of it), whatever the launch size; otherwise they could
    fill the GPU and wait for bulk rows that no resident block claims.  A short
    spin limit turns such a deadlock into an error within seconds."""
    torch = _torch()
    mats = [synth.circuit(400 + (q % 7) * 50, seed=900 + q) for q in range(700)]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], 4, solve_seq_rows=8, spin_limit=1 << 22)
    assert min(_nseg(bs.h, 8)) > 2000
    k = len(mats)
    vals = [[m.val if v == 0 else synth.circuit_values(m.rowptr, m.col, 40 + v * 1000 + q)
             for q, m in enumerate(mats)] for v in range(4)]
    bs.factor(torch.from_numpy(bs.concat_values(vals)).cuda())
    b = np.random.default_rng(6).standard_normal((2, bs.n))
    for _ in range(2):
        x = bs.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert bs.get_info().device_status == 0
    for q in range(0, 4 * k, 97):
        v, sidx = divmod(q, k)
        m = mats[sidx]
        rb = bs.row_base[q]
        for r in range(2):
            assert oracle.backward_error(m.n, m.rowptr, m.col, vals[v][sidx], x[r, rb:rb + m.n],
                                         b[r, rb:rb + m.n]) <= 1e-12
    bs.close()


def test_long_row_chunks_keep_the_level_order():
    """Long forward rows (2048+ L entries) are summed in chunks by other warps.
    On this 3D grid some long rows draw every entry from levels two or more
    below their own: such a row must still wait for its level before its
    node completes and raises the level watermark (otherwise the watermark
    could pass levels that are not complete, and later fall back).  Repeated
    one-right-hand-side solves (chunks) against a two-right-hand-side solve
    (whole rows) of the same factors; a short spin limit turns a stall into
    an error within seconds."""
    torch = _torch()
    A = synth.convdiff3d(40)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1, spin_limit=1 << 22)
    S = capi.hylu_export_solve_segments(s.h, 0, s.get_info().solve_seq_rows)
    sn = s.export_perm()[4]
    rp, ci = s.export_pattern()
    node_of = np.repeat(np.arange(len(sn) - 1), np.diff(sn))
    import sys
    sys.path.insert(0, __file__.rsplit("/", 1)[0])
    from plan_image import PlanImage
    lev = PlanImage(capi.hylu_plan_save(s.h)).fwd_level
    early = [r for r in np.unique(S["chunk_row"])
             if S["chunk_level"][S["row_chunk_off"][r]:S["row_chunk_off"][r + 1]].max() < lev[node_of[r]]]
    assert len(early) > 0, "no long row draws only from lower levels: the case tests nothing"
    s.factor(torch.from_numpy(A.val).cuda())
    _, b = synth.rhs(A, 21, 2)
    db = torch.from_numpy(b).cuda()
    x2 = s.solve(db).cpu().numpy().reshape(2, A.n)
    for _ in range(8):
        x1 = s.solve(db[0].clone()).cpu().numpy()
        assert s.get_info().device_status == 0
        assert oracle.backward_error(A.n, A.rowptr, A.col, A.val, x1, b[0]) <= 1e-12
        assert np.linalg.norm(x1 - x2[0]) <= 1e-12 * np.linalg.norm(x2[0])
    s.close()
