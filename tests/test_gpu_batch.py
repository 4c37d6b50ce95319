"""Batched form on the GPU: many value sets of one pattern and many patterns
of uneven size factored in one persistent launch (block-diagonal combined
plan), replayed from a CUDA graph.  Every instance is compared with the CPU
oracle run on that instance's own preprocessing outputs: padded pattern,
supernode partition and pivot order exactly, factors within 1e-10
normwise, and every solve to backward error <= 1e-12 (the graph with its
fixed FP64 refinement steps too)."""
import numpy as np
import pytest

import oracle
from paper_2509_07690_gb300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _systems():
    sizes = [700, 2000, 150, 3100, 1200]
    mats = [synth.circuit(n, seed=500 + q) for q, n in enumerate(sizes)]
    mats.append(synth.grid5(20))
    return mats


def _be(A, vals, x, b):
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ax = np.bincount(rid, weights=vals * x[A.col], minlength=A.n)
    an = np.bincount(rid, weights=np.abs(vals), minlength=A.n).max()
    return np.abs(b - ax).max() / (an * np.abs(x).max() + np.abs(b).max())


def test_batch_matches_oracle_and_graph_replay():
    torch = _torch()
    from paper_2509_07690_gb300 import BatchSolver
    mats = _systems()
    nsets = 3
    value_sets = [[m.val if v == 0 else synth.circuit_values(m.rowptr, m.col, 90 + 10 * v + q)
                   for q, m in enumerate(mats)] for v in range(nsets)]
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], nsets)
    k = len(mats)
    vals = torch.from_numpy(bs.concat_values(value_sets)).cuda()
    bs.factor(vals)
    gv, gpiv = bs.export_factors()
    prp, pci = bs.export_pattern()
    rp, cp, dr, dc, sn = bs.export_perm()
    rng = np.random.default_rng(8)
    nrhs = 2
    b = rng.standard_normal((nrhs, bs.n))
    db = torch.from_numpy(b).cuda()
    x = bs.solve(db).cpu().numpy()
    for v in range(nsets):
        for q, m in enumerate(mats):
            inst = v * k + q
            rb = bs.row_base[inst]
            sl = slice(rb, rb + m.n)
            o = oracle.Oracle(m.n, m.rowptr, m.col, value_sets[v][q], rp[sl] - rb, cp[sl] - rb, dr[sl], dc[sl])
            ov, opiv, _ = o.factors()
            lo, hi = prp[rb], prp[rb + m.n]
            assert np.array_equal(prp[rb:rb + m.n + 1] - lo, o.padded.rowptr)
            assert np.array_equal(pci[lo:hi] - rb, o.padded.col)
            inst_sn = sn[(sn >= rb) & (sn <= rb + m.n)] - rb
            assert np.array_equal(inst_sn, o.sn_start)
            assert np.array_equal(gpiv[sl] - rb, opiv)
            rel = np.linalg.norm(gv[lo:hi] - ov) / np.linalg.norm(ov)
            assert rel <= 1e-10, (v, q, rel)
            for r in range(nrhs):
                assert _be(m, value_sets[v][q], x[r, sl], b[r, sl]) <= 1e-12
    # one graph: refactor + solve, replayed on a created stream
    best = bs.tune(vals)
    assert 1 <= best <= 4
    ti = bs.get_info()
    assert ti.tuned == 1 and ti.factor_blocks_per_sm == best and 1 <= ti.solve_blocks_per_sm <= 4
    dx = torch.empty_like(db)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        # two fixed FP64 refinement steps inside the graph: 1e-12 holds
        # whether or not a replay perturbs a pivot
        bs.graph_capture(vals, db, dx, corrections=2, stream=side)
        for _ in range(2):
            dx.zero_()
            bs.graph_launch(stream=side)
            side.synchronize()
            xg = dx.cpu().numpy()
            info = bs.get_info()
            assert info.refine_iters == 2 and 0 <= info.backward_error <= 1e-12
            bound = 1e-12
            for v in range(nsets):
                for q, m in enumerate(mats):
                    rb = bs.row_base[v * k + q]
                    for r in range(nrhs):
                        assert _be(m, value_sets[v][q], xg[r, rb:rb + m.n], b[r, rb:rb + m.n]) <= bound
        # new values in the captured buffer: a replay that skipped a wait
        # would reuse the previous replay's factors
        new_sets = [[synth.circuit_values(m.rowptr, m.col, 300 + 10 * v + q) if q < k - 1 else 2.0 * m.val
                     for q, m in enumerate(mats)] for v in range(nsets)]
        vals.copy_(torch.from_numpy(bs.concat_values(new_sets)).cuda())
        dx.zero_()
        bs.graph_launch(stream=side)
        side.synchronize()
        xg = dx.cpu().numpy()
        info = bs.get_info()
        assert info.refine_iters == 2 and 0 <= info.backward_error <= 1e-12
        bound = 1e-12
        for v in range(nsets):
            for q, m in enumerate(mats):
                rb = bs.row_base[v * k + q]
                for r in range(nrhs):
                    assert _be(m, new_sets[v][q], xg[r, rb:rb + m.n], b[r, rb:rb + m.n]) <= bound
    bs.close()


def test_graph_refinement_reaches_1e12_with_perturbed_pivots():
    """Instances whose diagonal blocks carry exact zero pivots (perturbed to
    tau): the solve alone misses 1e-12; two recorded corrections reach it."""
    torch = _torch()
    from paper_2509_07690_gb300 import BatchSolver
    mats = []
    for q in range(4):
        # rows 0..2: [[0, 0, 1], [0, 1, 0], [1, 0, 1]] (stored zero diagonal;
        # row 0 is a standalone row, never pivoted, so its zero pivot is
        # perturbed), then a diagonally dominant tridiagonal block
        m = 24 + 7 * q
        r = [0, 0, 1, 2, 2]
        c = [0, 2, 1, 0, 2]
        v = [0.0, 1.0, 1.0, 1.0, 1.0]
        for i in range(3, m):
            for j, a in ((i - 1, -1.0), (i, 4.0 + 0.1 * q), (i + 1, -1.0)):
                if 3 <= j < m:
                    r.append(i); c.append(j); v.append(a)
        mats.append(synth.from_coo(m, np.array(r), np.array(c), np.array(v)))
    bs = BatchSolver([(m.n, m.rowptr, m.col, m.val) for m in mats], 1, static_pivot=0, ordering=2)
    vals = torch.from_numpy(bs.concat_values([[m.val for m in mats]])).cuda()
    bs.factor(vals)
    b = np.random.default_rng(2).standard_normal(bs.n)
    db = torch.from_numpy(b).cuda()
    bs.solve(db)
    assert bs.get_info().nperturb > 0
    dx = torch.empty_like(db)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        bs.graph_capture(vals, db, dx, corrections=0, stream=side)
        bs.graph_launch(stream=side)
        side.synchronize()
        be0 = bs.get_info().backward_error
        bs.graph_capture(vals, db, dx, corrections=2, stream=side)
        bs.graph_launch(stream=side)
        side.synchronize()
        info = bs.get_info()
    assert info.nperturb > 0 and be0 > 1e-12
    assert info.refine_iters == 2 and info.backward_error <= 1e-12
    xg = dx.cpu().numpy()
    for q, m in enumerate(mats):
        rb = bs.row_base[q]
        assert _be(m, m.val, xg[rb:rb + m.n], b[rb:rb + m.n]) <= 1e-12
    bs.close()
