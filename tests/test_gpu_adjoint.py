"""Differentiation form on the GPU: transpose solve against the CPU oracle,
gradients of L = w . x against a dense gradient and central finite
differences (Sec. 2.3 substitution reused by the adjoint)."""
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


def _be_transpose(A, y, g):
    at = A.todense().T
    r = g - at @ y
    return np.abs(r).max() / (np.abs(at).sum(1).max() * np.abs(y).max() + np.abs(g).max())


@pytest.mark.parametrize("case", ["grid5_20", "circuit_800", "convdiff_8_nd", "dense_60"])
def test_transpose_solve_matches_oracle(case):
    torch = _torch()
    from paper_2509_07690_gb300 import Solver
    opts = {}
    if case == "grid5_20":
        A = synth.grid5(20)
    elif case == "circuit_800":
        A = synth.circuit(800, seed=9)
    elif case == "convdiff_8_nd":
        A, opts = synth.convdiff3d(8), {"ordering": 1}
    else:
        rng = np.random.default_rng(60)
        a = rng.standard_normal((60, 60))
        r, c = np.nonzero(a)
        A = synth.from_coo(60, r, c, a[r, c])
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    s.factor(torch.from_numpy(A.val).cuda())
    rp, cp, dr, dc, _ = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc)
    g = np.random.default_rng(3).standard_normal((2, A.n))
    y = s.solve(torch.from_numpy(g).cuda(), transpose=True).cpu().numpy()
    for k in range(2):
        yo = o.solve_transpose(g[k])
        assert np.abs(y[k] - yo).max() <= 1e-9 * max(1.0, np.abs(yo).max())
        assert _be_transpose(A, y[k], g[k]) <= 1e-12
    s.close()


def _grad_case(A, opts, rng):
    torch = _torch()
    from paper_2509_07690_gb300 import Solver, solve
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    vals = torch.from_numpy(A.val.copy()).cuda().requires_grad_(True)
    xt, b = synth.rhs(A, 5)
    bt = torch.from_numpy(b[0]).cuda().requires_grad_(True)
    w = torch.from_numpy(rng.standard_normal(A.n)).cuda()
    x = solve(vals, bt, s)
    loss = (w * x).sum()
    loss.backward()
    return s, vals.grad.cpu().numpy(), bt.grad.cpu().numpy(), w.cpu().numpy(), b[0], x.detach().cpu().numpy()


def test_two_solves_on_one_solver_before_backward():
    """Two differentiable solves with different values on one Solver, then
    one backward: each gradient must be the dense-formula gradient of its
    own A, although the handle holds the second A's factors at backward."""
    torch = _torch()
    from paper_2509_07690_gb300 import Solver, solve
    A = synth.aniso9(10, seed=5)
    rng = np.random.default_rng(8)
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1)
    v1 = A.val.copy()
    v2 = A.val * rng.uniform(0.5, 1.5, A.nnz)
    b = rng.standard_normal(A.n)
    w1, w2 = rng.standard_normal(A.n), rng.standard_normal(A.n)
    t1 = torch.from_numpy(v1).cuda().requires_grad_(True)
    t2 = torch.from_numpy(v2).cuda().requires_grad_(True)
    bt = torch.from_numpy(b).cuda()
    x1 = solve(t1, bt, s)
    x2 = solve(t2, bt, s)
    loss = (torch.from_numpy(w1).cuda() * x1).sum() + (torch.from_numpy(w2).cuda() * x2).sum()
    loss.backward()
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    for vals, w, t in ((v1, w1, t1), (v2, w2, t2)):
        a = synth.CSR(A.n, A.rowptr, A.col, vals).todense()
        lam = np.linalg.solve(a.T, w)
        xd = np.linalg.solve(a, b)
        np.testing.assert_allclose(t.grad.cpu().numpy(), -lam[rid] * xd[A.col], rtol=1e-9, atol=1e-12)
    s.close()


@pytest.mark.parametrize("n_grid", [6, 12])
def test_gradient_matches_dense_formula(n_grid):
    rng = np.random.default_rng(n_grid)
    A = synth.aniso9(n_grid, seed=77)
    s, gA, gb, w, b, x = _grad_case(A, {"ordering": 1}, rng)
    a = A.todense()
    lam = np.linalg.solve(a.T, w)                    # dL/db
    xd = np.linalg.solve(a, b)
    np.testing.assert_allclose(gb, lam, rtol=1e-9, atol=1e-12)
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    np.testing.assert_allclose(gA, -lam[rid] * xd[A.col], rtol=1e-9, atol=1e-12)
    s.close()


def test_gradient_finite_differences_small():
    """Central differences of L(A, b) = w . A^{-1} b computed by the CPU oracle."""
    rng = np.random.default_rng(1)
    A = synth.circuit(400, seed=21)
    s, gA, gb, w, b, _ = _grad_case(A, {}, rng)
    rp, cp, dr, dc, _ = s.export_perm()

    def loss(vals, bb):
        o = oracle.Oracle(A.n, A.rowptr, A.col, vals, rp, cp, dr, dc)
        x, _, _ = o.solve_refine(bb, force=True)
        return float(w @ x)

    for q in rng.choice(A.nnz, 16, replace=False):
        h = 1e-6 * max(abs(A.val[q]), 1.0)
        vp, vm = A.val.copy(), A.val.copy()
        vp[q] += h
        vm[q] -= h
        fd = (loss(vp, b) - loss(vm, b)) / (2 * h)
        assert abs(fd - gA[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, gA[q])
    for k in rng.choice(A.n, 16, replace=False):
        h = 1e-6 * max(abs(b[k]), 1.0)
        bp, bm = b.copy(), b.copy()
        bp[k] += h
        bm[k] -= h
        fd = (loss(A.val, bp) - loss(A.val, bm)) / (2 * h)
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gb[k])
    s.close()


@pytest.mark.slow
def test_gradient_finite_differences_aniso_512():
    """Differentiation workload at full size: 2D 9-point anisotropic diffusion
    512x512, loss w . x; 64 entries of A and 64 components of b checked by
    central finite differences, each refactoring / re-solving on the GPU.
    The rounding noise of a difference quotient is about eps * cond(A) / h, so
    the steps are taken as large as the truncation error allows: L is linear
    in b (exact for any step, h = max(|b_k|, 1)); for entries of A the central
    differences at h and h/2 (h = 1e-3 max(|a|, 1)) are combined by Richardson
    extrapolation, leaving an O(h^4) truncation error."""
    torch = _torch()
    rng = np.random.default_rng(4)
    A = synth.workload("aniso9_512")
    s, gA, gb, w, b, _ = _grad_case(A, {"ordering": 1}, rng)
    dw = torch.from_numpy(w).cuda()
    db = torch.from_numpy(b).cuda()

    def loss(vals):
        s.factor(torch.from_numpy(vals).cuda())
        return float((dw * s.solve(db)).sum().item())

    def central(q, h):
        vp, vm = A.val.copy(), A.val.copy()
        vp[q] += h
        vm[q] -= h
        return (loss(vp) - loss(vm)) / (2 * h)

    for q in rng.choice(A.nnz, 64, replace=False):
        h = 1e-3 * max(abs(A.val[q]), 1.0)
        fd = (4.0 * central(q, h / 2) - central(q, h)) / 3.0
        assert abs(fd - gA[q]) <= 1e-6 * max(1.0, abs(fd)), ("A", q, fd, gA[q])
    s.factor(torch.from_numpy(A.val).cuda())
    for k in rng.choice(A.n, 64, replace=False):
        h = max(abs(b[k]), 1.0)
        bp, bm = b.copy(), b.copy()
        bp[k] += h
        bm[k] -= h
        x = s.solve(torch.from_numpy(np.stack([bp, bm])).cuda()).cpu().numpy()
        fd = (w @ x[0] - w @ x[1]) / (2 * h)
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(fd)), ("b", k, fd, gb[k])
    s.close()
