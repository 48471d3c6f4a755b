"""The tensor-core product on E4M3 operands (tcgen05 kind::f8f6f4) through the C
ABI, against a plain FP64 product of the same E4M3 values.

This is the product of the batched solver when X is stored in FP8 e4m3 with
power-of-two column scales: KSC_E4M3_PIECES E4M3 pieces of each vector row, the row scaled
by a power of two, against E4M3 X; the first three pieces and the last two (a
remainder scaled by 2^12) accumulate separately and are added as hi + 2^-12 lo;
the epilogue multiplies row i by its inverse scale and column j by the column
scale.  Products of E4M3 values are exact in
FP32 and the scales are powers of two, so only the FP32 accumulation rounds:
|D - D_ref| <= (K' + 2) u_32 sum |a||b| with K' = pieces x k.  A descriptor or layout
mistake (a wrong K step of 32 bytes, a transposed or shifted operand, a lost
piece, a scale on the wrong axis) gives errors of the size of the entries.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
PIECES = None   # the library's KSC_E4M3_PIECES, read in the fixture


@pytest.fixture(scope="module")
def K():
    global PIECES
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    PIECES = ksc.KSC_E4M3_PIECES
    return ksc


def _e4m3(x):
    """E4M3 (round to nearest) of a float tensor: (bytes, values as float64)."""
    q = x.to(torch.float8_e4m3fn)
    return q.view(torch.uint8), q.to(torch.float64)


def _run(K, m, m_pad, k, lda, n, ldb, tile_n, grid, seed, with_cs=True):
    gen = torch.Generator().manual_seed(seed)
    A = torch.randn(PIECES, m_pad, lda, generator=gen) * 64.0
    for q in range(1, PIECES):          # later pieces smaller, like a split vector
        A[q] *= 2.0 ** (-4 * q)
    B = torch.randn(n, ldb, generator=gen) * 16.0
    Ab, Av = _e4m3(A)
    Bb, Bv = _e4m3(B)
    rs = torch.tensor(np.ldexp(1.0, np.random.default_rng(seed).integers(-12, 4, m)), dtype=torch.float32)
    cs = torch.tensor(np.ldexp(1.0, np.random.default_rng(seed + 1).integers(-8, 2, n)), dtype=torch.float32)
    ldd = (n + 3) // 4 * 4
    Ad, Bd, rsd, csd = Ab.cuda(), Bb.cuda(), rs.cuda(), cs.cuda()
    D = torch.full((m, ldd), float("nan"), device="cuda", dtype=torch.float32)
    K.ksc_tc_gemm_e4m3(Ad.data_ptr(), m, m_pad, k, lda, Bd.data_ptr(), n, ldb, rsd.data_ptr(),
                       csd.data_ptr() if with_cs else 0, D.data_ptr(), ldd, tile_n, grid)
    torch.cuda.synchronize()
    a = Av[:, :m, :k]
    b = Bv[:, :k]
    w = [1.0 if q < 3 else 2.0 ** -12 for q in range(PIECES)]   # the low pieces' accumulator
    ref = sum(w[q] * (a[q] @ b.T) for q in range(PIECES))
    mag = sum(w[q] * (a[q].abs() @ b.abs().T) for q in range(PIECES))
    sc = rs.double()[:, None] * (cs.double()[None, :] if with_cs else 1.0)
    return D[:, :n].double().cpu(), ref * sc, mag * sc


CASES = [
    # m, m_pad, k, lda, n, ldb, tile_n, grid
    (128, 128, 128, 128, 64, 128, 64, 0),
    (200, 256, 1000, 1008, 300, 1008, 128, 0),
    (512, 512, 4000, 4000, 1000, 4000, 128, 0),
    (1, 128, 40, 48, 17, 48, 64, 0),
    (384, 384, 3000, 3008, 777, 3008, 128, 152),
    (1000, 1024, 2000, 2000, 530, 2000, 128, 152),
    (128, 128, 5000, 5008, 200, 5008, 64, 7),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "m{}k{}n{}bn{}g{}".format(c[0], c[2], c[4], c[6], c[7]))
def test_e4m3_product_matches_fp64(K, case):
    m, m_pad, k, lda, n, ldb, tile_n, grid = case
    got, ref, mag = _run(K, *case, seed=sum(case))
    assert torch.isfinite(got).all()
    bound = (PIECES * k + 2) * U32 * mag + 1e-30
    err = (got - ref).abs()
    assert (err <= bound).all(), float((err / bound).max())


def test_e4m3_product_without_column_scales(K):
    got, ref, mag = _run(K, 256, 256, 700, 704, 300, 704, 128, 0, seed=5, with_cs=False)
    assert ((got - ref).abs() <= (PIECES * 700 + 2) * U32 * mag + 1e-30).all()


def test_e4m3_product_rejects_bad_shapes(K):
    A = torch.zeros(PIECES * 128, 128, dtype=torch.uint8, device="cuda")   # pieces x m_pad rows
    B = torch.zeros(64, 128, dtype=torch.uint8, device="cuda")
    rs = torch.ones(128, dtype=torch.float32, device="cuda")
    D = torch.zeros(128, 64, dtype=torch.float32, device="cuda")
    with pytest.raises(K.KscError):   # row stride not a multiple of 16 bytes
        K.ksc_tc_gemm_e4m3(A.data_ptr(), 128, 128, 100, 100, B.data_ptr(), 64, 128, rs.data_ptr(), 0,
                           D.data_ptr(), 64, 64, 0)
    with pytest.raises(K.KscError):   # m_pad not a multiple of 128
        K.ksc_tc_gemm_e4m3(A.data_ptr(), 100, 100, 128, 128, B.data_ptr(), 64, 128, rs.data_ptr(), 0,
                           D.data_ptr(), 64, 64, 0)
    with pytest.raises(K.KscError):   # tiles wider than 128 (two accumulators)
        K.ksc_tc_gemm_e4m3(A.data_ptr(), 128, 128, 128, 128, B.data_ptr(), 64, 128, rs.data_ptr(), 0,
                           D.data_ptr(), 64, 256, 0)
    with pytest.raises(K.KscError):   # no row scales
        K.ksc_tc_gemm_e4m3(A.data_ptr(), 128, 128, 128, 128, B.data_ptr(), 64, 128, 0, 0,
                           D.data_ptr(), 64, 64, 0)
