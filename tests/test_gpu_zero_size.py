"""The empty system on the GPU: n = 0 is analysed to an empty plan, and
factorization, refactorization and both solves (one and several right-hand
sides) accept empty CUDA tensors, return HYLU_OK and launch no kernel."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_empty_system_factor_and_solves_launch_nothing():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_07690_gb300 import Solver, capi
    s = Solver(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    l0 = capi.hylu_launch_count()
    assert s.factor(empty) == 0
    assert s.factor(empty) == 0                      # refactorization
    x = s.solve(empty)
    assert x.is_cuda and tuple(x.shape) == (0,)
    b = torch.empty(3, 0, dtype=torch.float64, device="cuda")
    x = s.solve(b, transpose=True)
    assert tuple(x.shape) == (3, 0)
    torch.cuda.synchronize()
    assert capi.hylu_launch_count() == l0
    info = s.get_info()
    assert info.n == 0 and info.nnodes == 0 and info.device_status == 0
    s.close()
