"""hylu_solve_static, the substitution that allocates nothing, against
hylu_solve.

Some callers cannot let this library allocate device memory for them: a
program whose own pool already holds the device memory, or a loop that
cannot absorb the device-wide synchronization of cudaMalloc.
hylu_solve_static serves them from a fixed array compiled into the library.
On the same factors it must give hylu_solve's solution (no pivot is perturbed
in these cases, so hylu_solve does not refine) on consecutive calls that reuse
the shared array.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _backward_error(A, x, b):
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ax = np.bincount(rid, weights=A.val * x[A.col], minlength=A.n)
    anorm = np.bincount(rid, weights=np.abs(A.val), minlength=A.n).max()
    return np.abs(b - ax).max() / (anorm * np.abs(x).max() + np.abs(b).max())


@pytest.mark.parametrize("case", ["grid5_40_amd", "convdiff3d_10_nd"])
def test_static_solve_matches_solve(case):
    torch = _torch()
    from paper_2509_07690_gb300 import Solver, capi, synth
    if case == "grid5_40_amd":
        A, opts = synth.grid5(40), {}
    else:
        A, opts = synth.convdiff3d(10), {"ordering": 1}
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    s.factor(torch.from_numpy(A.val).cuda())
    assert s.get_info().nperturb == 0
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(11)
    for _ in range(2):                      # two calls in a row share the array
        b_host = rng.standard_normal(A.n)
        b = torch.from_numpy(b_host).cuda()
        ref = s.solve(b).cpu().numpy()
        x = torch.full_like(b, float("nan"))
        capi.hylu_solve_static(s.h, b.data_ptr(), x.data_ptr(), stream)
        torch.cuda.synchronize()
        got = x.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        assert _backward_error(A, got, b_host) <= 1e-12
    s.close()


def test_static_solve_rejects_n_above_limit():
    torch = _torch()
    from paper_2509_07690_gb300 import Solver, capi
    n = capi.HYLU_STATIC_SOLVE_MAX_N + 1
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    s = Solver(n, rp, ci, np.ones(n), static_pivot=0, ordering=2)
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(capi.HyluError) as err:
        capi.hylu_solve_static(s.h, b.data_ptr(), x.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert err.value.code == capi.HYLU_ERR_TOO_LARGE
    s.close()


def test_static_solve_first_on_fresh_handle_allocates_nothing():
    """The allocation-free call as the first substitution of a newly factored
    handle (its hylu_solve work vectors do not exist yet): device free memory
    is unchanged across the call, and the result equals a later hylu_solve.
    A warm-up handle first makes the array's module resident, so the
    measurement sees only what the call itself would allocate."""
    torch = _torch()
    from paper_2509_07690_gb300 import Solver, capi, synth
    stream = torch.cuda.current_stream().cuda_stream
    A = synth.grid5(30)
    warm = Solver(A.n, A.rowptr, A.col, A.val)
    warm.factor(torch.from_numpy(A.val).cuda())
    bw = torch.ones(A.n, dtype=torch.float64, device="cuda")
    xw = torch.empty_like(bw)
    capi.hylu_solve_static(warm.h, bw.data_ptr(), xw.data_ptr(), stream)
    torch.cuda.synchronize()

    B = synth.convdiff3d(9)
    s = Solver(B.n, B.rowptr, B.col, B.val, ordering=1)
    s.factor(torch.from_numpy(B.val).cuda())
    b_host = np.random.default_rng(4).standard_normal(B.n)
    b = torch.from_numpy(b_host).cuda()
    x = torch.full_like(b, float("nan"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    capi.hylu_solve_static(s.h, b.data_ptr(), x.data_ptr(), stream)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    assert s.get_info().nperturb == 0
    ref = s.solve(b).cpu().numpy()
    got = x.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    assert _backward_error(B, got, b_host) <= 1e-12
    warm.close()
    s.close()


def test_static_solve_refuses_fp32_factors_and_accepts_empty_system():
    torch = _torch()
    from paper_2509_07690_gb300 import Solver, capi, synth
    stream = torch.cuda.current_stream().cuda_stream
    A = synth.grid5(12)
    s = Solver(A.n, A.rowptr, A.col, A.val, precision=1)
    s.factor(torch.from_numpy(A.val).cuda())
    b = torch.ones(A.n, dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    with pytest.raises(capi.HyluError) as err:
        capi.hylu_solve_static(s.h, b.data_ptr(), x.data_ptr(), stream)
    assert err.value.code == capi.HYLU_ERR_STATE
    s.close()
    e = Solver(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    e.factor(empty)
    assert capi.hylu_solve_static(e.h, 0, 0, stream) == 0
    e.close()
