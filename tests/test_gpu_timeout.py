"""Failure detection on the GPU without a fault: every device wait is bounded.
A handle analysed with a spin limit of one iteration makes the factor
kernel's first wait on a not yet finished row run out; the kernel records
HYLU_ERR_DEVICE_TIMEOUT, every warp leaves, and the context stays usable (a
second handle factors and solves the same matrix correctly)."""
import numpy as np
import pytest

import oracle
from paper_2509_07690_gb300 import capi, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _chain(n):
    # tridiagonal, diagonally dominant: in natural order every row waits on
    # the row before it
    r = np.concatenate([np.arange(n - 1), np.arange(1, n), np.arange(n)])
    c = np.concatenate([np.arange(1, n), np.arange(n - 1), np.arange(n)])
    v = np.concatenate([-np.ones(n - 1), -np.ones(n - 1), 4.0 * np.ones(n)])
    return synth.from_coo(n, r, c, v)


def test_expired_wait_reports_timeout_and_context_survives():
    torch = _torch()
    from paper_2509_07690_gb300 import Solver
    A = _chain(20000)
    d = torch.from_numpy(A.val).cuda()
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=2, static_pivot=0, sn_max=1, spin_limit=1)
    s.factor(d)
    with pytest.raises(capi.HyluError) as e:
        s.get_info()
    assert e.value.code == -6                      # HYLU_ERR_DEVICE_TIMEOUT
    s.close()
    torch.cuda.synchronize()
    ok = Solver(A.n, A.rowptr, A.col, A.val, ordering=2, static_pivot=0, sn_max=1)
    ok.factor(d)
    xt, b = synth.rhs(A, 11)
    x = ok.solve(torch.from_numpy(b[0]).cuda()).cpu().numpy()
    assert ok.get_info().device_status == 0
    assert oracle.backward_error(A.n, A.rowptr, A.col, A.val, x, b[0]) <= 1e-12
    ok.close()
