"""The tensor-core tile engine of the precision form's sup-sup update (HYLU
Sec. 2.2, Fig. 1c: supernode-to-supernode updates as dense products), on
plain dense matrices through the C ABI: C -= A B with FP32 operands split
into BF16 terms, tcgen05 MMAs and FP32 accumulation in tensor memory.
Checked elementwise against the FP64 product of the same FP32 inputs.

Error bound per entry, from the splitting: an FP32 value x is carried as
nsplit BF16 terms whose remainder is at most 2^(-8 nsplit) |x|, and the
dropped term products are of the same order, so the product error is at
most about 3 * 2^(-8 nsplit) (|A| |B|)_ij plus the FP32 accumulation
(2^-24 per addition over k terms).  The tests allow
  |err_ij| <= (4 * 2^(-8 nsplit) + k * 2^-23) (|A| |B|)_ij + 2^-23 |C_ij|."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(m, n, k, nsplit, seed, scale_rows=False):
    torch = _torch()
    from paper_2509_07690_gb300 import capi
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, k)).astype(np.float32)
    if scale_rows:
        a *= np.exp(rng.uniform(-8, 8, (m, 1))).astype(np.float32)
    b = rng.standard_normal((k, n)).astype(np.float32)
    c = rng.standard_normal((m, n)).astype(np.float32)
    da, db, dc = (torch.from_numpy(x).cuda() for x in (a, b, c))
    capi.hylu_split_gemm(da.data_ptr(), db.data_ptr(), dc.data_ptr(), m, n, k, k, n, n, nsplit,
                         torch.cuda.current_stream().cuda_stream)
    got = dc.cpu().numpy().astype(np.float64)
    want = c.astype(np.float64) - a.astype(np.float64) @ b.astype(np.float64)
    mag = np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64))
    bound = (4.0 * 2.0 ** (-8 * nsplit) + k * 2.0 ** -23) * mag + 2.0 ** -23 * np.abs(c)
    err = np.abs(got - want)
    assert np.all(np.isfinite(got))
    worst = float(np.max(err / np.maximum(bound, 1e-300)))
    assert np.all(err <= bound), (worst, float(err.max()))
    return float(np.max(err / np.maximum(mag, 1e-300)))


@pytest.mark.parametrize("shape", [(128, 64, 32), (200, 100, 75), (384, 192, 256), (1, 1, 1), (130, 65, 33),
                                   (256, 320, 700)])
@pytest.mark.parametrize("nsplit", [2, 3])
def test_split_gemm_matches_fp64_product(shape, nsplit):
    m, n, k = shape
    _run(m, n, k, nsplit, seed=m + 7 * n + 13 * k + nsplit)


def _single_products(nsplit):
    """Relative error of single products (k = 1, C = 0): no accumulation, so
    what is left is the splitting and one FP32 rounding of the result."""
    torch = _torch()
    from paper_2509_07690_gb300 import capi
    rng = np.random.default_rng(23)
    m, n = 256, 128
    a = rng.uniform(0.5, 2.0, (m, 1)).astype(np.float32)
    b = rng.uniform(0.5, 2.0, (1, n)).astype(np.float32)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dc = torch.zeros((m, n), dtype=torch.float32, device="cuda")
    capi.hylu_split_gemm(da.data_ptr(), db.data_ptr(), dc.data_ptr(), m, n, 1, 1, n, n, nsplit,
                         torch.cuda.current_stream().cuda_stream)
    want = -(a.astype(np.float64) @ b.astype(np.float64))
    return float(np.max(np.abs(dc.cpu().numpy() - want) / np.abs(want)))


def test_three_terms_are_more_accurate_than_two():
    # two terms drop the product of the second terms (up to ~2^-17 of the
    # product); with three terms what is left is the accumulation of the six
    # term products inside the tensor core, whose FP32 sums are not rounded
    # to nearest: measured ~4e-7 (about 2^-21) relative on GB300
    e2 = _single_products(2)
    e3 = _single_products(3)
    assert 2.0 ** -21 < e2 <= 2.0 ** -15
    assert e3 <= 2.0 ** -20
    assert e3 < e2 / 4


def test_rows_of_very_different_magnitude():
    # the splitting is relative to each value: rows scaled by e^-8 .. e^8 keep
    # their relative accuracy
    _run(256, 64, 96, 3, seed=17, scale_rows=True)


def test_rejects_bad_sizes():
    torch = _torch()
    from paper_2509_07690_gb300 import capi
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = x.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    for args in ((4, 4, 4, 3, 4, 4, 3), (4, 4, 4, 4, 4, 4, 4), (-1, 4, 4, 4, 4, 4, 3)):
        m, n, k, lda, ldb, ldc, ns = args
        with pytest.raises(capi.HyluError) as e:
            capi.hylu_split_gemm(p, p, p, m, n, k, lda, ldb, ldc, ns, s)
        assert e.value.code == capi.HYLU_ERR_ARG
    assert capi.hylu_split_gemm(p, p, p, 0, 4, 4, 4, 4, 4, 3, s) == 0
