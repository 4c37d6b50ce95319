"""GPU at the configurations' full sizes, in the options bench.py times.

The oracle's numeric factorization does not finish at these sizes, so the
checks are what it can pin and what holds at any size: the symbolic pattern,
supernode partition and flop count bit-exact against the oracle's own
symbolic pass (circuit_100k, aniso9_512), and backward error <= 1e-12 of
every solve (refactored value sets, transpose solve, precision form)."""
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


def _pattern_matches_oracle(s, A):
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc, numeric=False)
    prp, pci = s.export_pattern()
    assert np.array_equal(o.sn_start, sn)
    assert np.array_equal(o.padded.rowptr, prp) and np.array_equal(o.padded.col, pci)
    assert s.info.flops == o.flops[0] and s.info.flops_padded == o.flops[1]


def _be(A, vals, x, b, transpose=False):
    return oracle.backward_error(A.n, A.rowptr, A.col, vals, x, b) if not transpose else _be_t(A, vals, x, b)


def _be_t(A, vals, x, b):
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    atx = np.bincount(A.col, weights=vals * x[rid], minlength=A.n)
    an = np.bincount(A.col, weights=np.abs(vals), minlength=A.n).max()
    return np.abs(b - atx).max() / (an * np.abs(x).max() + np.abs(b).max())


def test_circuit_100k_pattern_and_refactor():
    torch = _torch()
    from paper_2509_07690_gb300 import Solver
    A = synth.workload("circuit_100k")
    s = Solver(A.n, A.rowptr, A.col, A.val)
    _pattern_matches_oracle(s, A)
    xt, b = synth.rhs(A, 1002)
    db = torch.from_numpy(b[0]).cuda()
    for j in range(3):
        vals = A.val if j == 0 else synth.circuit_value_set(A, 1003 + j).val
        s.factor(torch.from_numpy(vals).cuda())
        x = s.solve(db).cpu().numpy()
        info = s.get_info()
        assert info.device_status == 0
        assert _be(A, vals, x, b[0]) <= 1e-12
    s.close()


def test_aniso9_512_pattern_solve_and_transpose():
    torch = _torch()
    from paper_2509_07690_gb300 import Solver
    A = synth.workload("aniso9_512")
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1)
    _pattern_matches_oracle(s, A)
    s.factor(torch.from_numpy(A.val).cuda())
    xt, b = synth.rhs(A, 1004, 3)
    x = s.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    for r in range(3):
        assert _be(A, A.val, x[r], b[r]) <= 1e-12
    y = s.solve(torch.from_numpy(b[0]).cuda(), transpose=True).cpu().numpy()
    assert _be_t(A, A.val, y, b[0]) <= 1e-12
    assert s.get_info().device_status == 0
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_convdiff3d_64_solve(precision):
    torch = _torch()
    from paper_2509_07690_gb300 import Solver
    A = synth.workload("convdiff3d_64")
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1, precision=precision)
    s.factor(torch.from_numpy(A.val).cuda())
    xt, b = synth.rhs(A, 1003, 8)
    x = s.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    info = s.get_info()
    assert info.device_status == 0
    for r in range(8):
        assert _be(A, A.val, x[r], b[r]) <= 1e-12, r
    if precision == 1:
        assert info.refine_iters >= 1
    s.close()
