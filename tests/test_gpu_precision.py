"""Precision form on the GPU: FP32 factors (scaling and the small-pivot check
in FP64) refined in FP64 to backward error <= 1e-12; the error of the FP32
factors against the FP64 oracle is measured and bounded."""
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


def _be(A, x, b):
    rid = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    ax = np.bincount(rid, weights=A.val * x[A.col], minlength=A.n)
    an = np.bincount(rid, weights=np.abs(A.val), minlength=A.n).max()
    return np.abs(b - ax).max() / (an * np.abs(x).max() + np.abs(b).max())


def _dense_lu(prp, pci, vals, piv, sn):
    """Dense (L, U) in position order from factors stored on the padded
    pattern (the layout hylu_export_factors documents)."""
    n = len(prp) - 1
    end_of = np.empty(n, np.int64)
    for q in range(len(sn) - 1):
        end_of[sn[q]:sn[q + 1]] = sn[q + 1] - 1
    pinv = np.empty(n, np.int64)
    pinv[piv] = np.arange(n)
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for t in range(prp[i], prp[i + 1]):
            c = int(pci[t])
            if c < i:
                L[i, c] = vals[t]
            else:
                U[i, c if c <= end_of[i] else pinv[c]] = vals[t]
    return L, U


@pytest.mark.parametrize("case", ["grid5_32", "convdiff_12_nd", "aniso_48_nd", "circuit_3000"])
def test_fp32_factors_refined_to_fp64_accuracy(case):
    torch = _torch()
    from paper_2509_07690_gb300 import Solver
    opts = {"precision": 1}
    if case == "grid5_32":
        A = synth.grid5(32)
    elif case == "convdiff_12_nd":
        A = synth.convdiff3d(12); opts["ordering"] = 1
    elif case == "aniso_48_nd":
        A = synth.aniso9(48); opts["ordering"] = 1
    else:
        A = synth.circuit(3000, seed=31)
    s = Solver(A.n, A.rowptr, A.col, A.val, **opts)
    s.factor(torch.from_numpy(A.val).cuda())
    rp, cp, dr, dc, sn = s.export_perm()
    o = oracle.Oracle(A.n, A.rowptr, A.col, A.val, rp, cp, dr, dc)
    ov, opiv, _ = o.factors()
    gv, gpiv = s.export_factors()
    prp, pci = s.export_pattern()
    assert np.array_equal(o.padded.col, pci)
    same = float(np.mean(opiv == gpiv))
    rel = np.linalg.norm(gv - ov) / np.linalg.norm(ov)
    # reconstruction of the FP32 factors: ||L U - Ahat[:, piv]||_F / ||Ahat||_F
    arp, aci, av = o.ahat
    ah = oracle.csr_dense(A.n, arp, aci, av)
    L, U = _dense_lu(prp, pci, gv, gpiv, sn)
    recon = np.linalg.norm(L @ U - ah[:, gpiv]) / np.linalg.norm(ah)
    eps32 = float(np.finfo(np.float32).eps)
    assert recon <= 64 * eps32, recon
    # where every pivot agrees, the factors themselves are within a modest
    # multiple of eps_32 of the FP64 oracle's (at a near-tie the FP32
    # elimination may pick the other entry: then the reconstruction above is
    # the check)
    if same == 1.0:
        assert rel <= 1e-4, rel
    xt, b = synth.rhs(A, 3, 2)
    x = s.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    info = s.get_info()
    assert info.refine_iters >= 1
    be = [_be(A, x[r], b[r]) for r in range(2)]
    for r in range(2):
        assert be[r] <= 1e-12
    # one line per case for the record of the form's error against FP64
    print(f"PRECISION_FORM case={case} n={A.n} pivots_equal={same:.4f} factor_rel_err={rel:.3e} "
          f"recon={recon:.3e} refine_iters={info.refine_iters} backward_error={max(be):.3e}")
    s.close()
