"""The circuit workload under nested dissection on the GPU (the ordering
bench.py times for it): hub rows ordered last, a dependency graph 6.4x
shallower than under AMD.

Parity against the oracle on circuits of 3,000 and 20,000 rows (at 20,000
the hub rows take the heavy-row queue): pattern and supernode partition bit
for bit, pivot order identical, factor values within 1e-10 normwise,
backward error <= 1e-12.  At full size (n = 100,000), where the oracle's
numeric factorization does not finish: pattern, partition and flop count
against the oracle's symbolic pass, and backward error <= 1e-12 for the
matrix and two refactored value sets."""
import numpy as np
import pytest

import oracle
from paper_2509_07690_gb300 import synth

from test_gpu_parity import run_case

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("n,seed", [(3000, 12), (20000, 77)])
def test_circuit_nested_dissection_parity(n, seed):
    run_case(synth.circuit(n, seed=seed), ordering=1)


def test_circuit_100k_nested_dissection():
    torch = _torch()
    from paper_2509_07690_gb300 import Solver
    A = synth.workload("circuit_100k")
    s = Solver(A.n, A.rowptr, A.col, A.val, ordering=1)
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc, numeric=False)
    prp, pci = s.export_pattern()
    assert np.array_equal(o.sn_start, sn)
    assert np.array_equal(o.padded.rowptr, prp) and np.array_equal(o.padded.col, pci)
    assert s.info.flops == o.flops[0] and s.info.flops_padded == o.flops[1]
    assert s.info.factor_levels < 2000                    # the shallow dependency graph
    _, b = synth.rhs(A, 1002)
    db = torch.from_numpy(b[0]).cuda()
    for j in range(3):
        vals = A.val if j == 0 else synth.circuit_value_set(A, 1003 + j).val
        s.factor(torch.from_numpy(vals).cuda())
        x = s.solve(db).cpu().numpy()
        assert s.get_info().device_status == 0
        assert oracle.backward_error(A.n, A.rowptr, A.col, vals, x, b[0]) <= 1e-12
    s.close()
