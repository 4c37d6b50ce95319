"""Warm start from a saved analysis: a solver loaded with Solver.load
(hylu_plan_load) from the image of an analysed one factors and solves the
same matrix like it: identical pivot order, factor values within 1e-12
normwise (reductions into shared rows may round in another order), backward
error <= 1e-12 for every right-hand side."""
import numpy as np
import pytest

from paper_2509_07690_gb300 import synth

pytestmark = pytest.mark.gpu


def _backward_error(A, x, b):
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ax = np.bincount(rid, weights=A.val * x[A.col], minlength=A.n)
    anorm = np.bincount(rid, weights=np.abs(A.val), minlength=A.n).max()
    return np.abs(b - ax).max() / (anorm * np.abs(x).max() + np.abs(b).max())


@pytest.mark.parametrize("case", ["circuit_3000", "convdiff3d_10_nd"])
def test_loaded_plan_factors_like_the_analysed_one(case, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07690_gb300 import Solver
    if case == "circuit_3000":
        A, opts = synth.circuit(3000, seed=21), {}
    else:
        A, opts = synth.convdiff3d(10), {"ordering": 1}
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    path = tmp_path / "plan.bin"
    s.save(path)
    t = Solver.load(path)
    d = torch.from_numpy(A.val).cuda()
    s.factor(d)
    t.factor(d)
    sv, spiv = s.export_factors()
    tv, tpiv = t.export_factors()
    assert np.array_equal(spiv, tpiv)
    assert np.linalg.norm(tv - sv) <= 1e-12 * np.linalg.norm(sv)
    _, b = synth.rhs(A, 7, nrhs=2)
    x = t.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    for r in range(2):
        assert _backward_error(A, x[r], b[r]) <= 1e-12
    assert t.get_info().device_status == 0
    s.close()
    t.close()
