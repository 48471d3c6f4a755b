"""The tensor-core product (tcgen05 + TMA + TMEM) through the C ABI, against a
plain FP64 product of the same BF16 operands.

The kernel's products of BF16 values are exact in FP32; only the FP32
accumulation rounds.  The bound used is the classical one for a sum of K' = k *
pieces products, |D - D_ref| <= (K' + 2) u_32 sum |a||b|, which every summation
order meets; a layout or descriptor mistake (a wrong K step, a transposed or
shifted operand, a lost piece) gives errors of the size of the entries themselves.
"""
import pytest
import torch

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


def _run(K, pieces, m, m_pad, k, lda, n, ldb, tile_n, seed, grid=0):
    gen = torch.Generator().manual_seed(seed)
    A = torch.randn(pieces, m_pad, lda, generator=gen).to(torch.bfloat16)
    B = torch.randn(n, ldb, generator=gen).to(torch.bfloat16)
    # later pieces carry smaller magnitudes, like the split of an FP32 vector
    for q in range(1, pieces):
        A[q] = (A[q].float() * 2.0 ** (-8 * q)).to(torch.bfloat16)
    ldd = (n + 3) // 4 * 4
    Ad, Bd = A.cuda(), B.cuda()
    D = torch.full((m, ldd), float("nan"), device="cuda", dtype=torch.float32)
    if grid:
        K.ksc_tc_gemm_sk(Ad.data_ptr(), pieces, m, m_pad, k, lda, Bd.data_ptr(), n, ldb, D.data_ptr(), ldd,
                         tile_n, grid)
    else:
        K.ksc_tc_gemm(Ad.data_ptr(), pieces, m, m_pad, k, lda, Bd.data_ptr(), n, ldb, D.data_ptr(), ldd,
                      tile_n)
    torch.cuda.synchronize()
    a = A[:, :m, :k].double()
    b = B[:, :k].double()
    ref = sum(a[q] @ b.T for q in range(pieces))
    mag = sum(a[q].abs() @ b.abs().T for q in range(pieces))
    got = D[:, :n].double().cpu()
    return got, ref, mag


CASES = [
    # pieces, m, m_pad, k, lda, n, ldb, tile_n
    (1, 128, 128, 64, 64, 64, 64, 64),
    (1, 128, 128, 1000, 1000, 300, 1000, 128),
    (3, 200, 256, 777, 784, 1000, 784, 256),
    (2, 512, 512, 5000, 5000, 1000, 5000, 128),
    (3, 384, 384, 2000, 2000, 777, 2008, 64),
    (1, 1, 128, 40, 40, 17, 40, 64),
    (3, 512, 512, 10000, 10000, 530, 10000, 256),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "P{}m{}k{}n{}bn{}".format(c[0], c[1], c[3], c[5], c[7]))
def test_tc_gemm_matches_fp64_product(K, case):
    pieces, m, m_pad, k, lda, n, ldb, tile_n = case
    got, ref, mag = _run(K, pieces, m, m_pad, k, lda, n, ldb, tile_n, seed=sum(case))
    assert torch.isfinite(got).all()
    bound = (k * pieces + 2) * U32 * mag + 1e-30
    err = (got - ref).abs()
    assert (err <= bound).all(), float((err / bound).max())


def test_tc_gemm_rejects_bad_shapes(K):
    A = torch.zeros(1, 128, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(64, 64, dtype=torch.bfloat16, device="cuda")
    D = torch.zeros(128, 64, dtype=torch.float32, device="cuda")
    with pytest.raises(K.KscError):   # m_pad not a multiple of 128
        K.ksc_tc_gemm(A.data_ptr(), 1, 100, 100, 64, 64, B.data_ptr(), 64, 64, D.data_ptr(), 64, 64)
    with pytest.raises(K.KscError):   # row stride not a multiple of 16 bytes
        K.ksc_tc_gemm(A.data_ptr(), 1, 128, 128, 60, 60, B.data_ptr(), 64, 64, D.data_ptr(), 64, 64)
    with pytest.raises(K.KscError):   # tile width
        K.ksc_tc_gemm(A.data_ptr(), 1, 128, 128, 64, 64, B.data_ptr(), 64, 64, D.data_ptr(), 64, 96)


# stream-K: tiles split over CTAs at any K block, partials summed by the fix-up
# kernel; grids from 1 (everything in one CTA, several tiles and both TMEM
# buffers) to more CTAs than K blocks (empty ranges, tiles spread over many CTAs)
SK_CASES = [
    # pieces, m, m_pad, k, lda, n, ldb, tile_n, grid
    (1, 128, 128, 640, 640, 300, 640, 64, 1),
    (3, 200, 256, 777, 784, 1000, 784, 256, 3),
    (3, 512, 512, 5000, 5000, 1000, 5000, 128, 152),
    (2, 384, 384, 2000, 2000, 777, 2008, 64, 7),
    (1, 1, 128, 40, 40, 17, 40, 64, 5),
    (3, 1024, 1024, 3000, 3000, 700, 3000, 256, 152),
    (3, 130, 256, 10000, 10000, 530, 10000, 128, 64),
    (1, 128, 128, 128, 128, 64, 128, 64, 400),
]


@pytest.mark.parametrize("case", SK_CASES, ids=lambda c: "P{}m{}k{}n{}bn{}g{}".format(c[0], c[1], c[3], c[5], c[7], c[8]))
def test_tc_gemm_stream_k_matches_fp64_product(K, case):
    pieces, m, m_pad, k, lda, n, ldb, tile_n, grid = case
    got, ref, mag = _run(K, pieces, m, m_pad, k, lda, n, ldb, tile_n, seed=sum(case), grid=grid)
    assert torch.isfinite(got).all()
    bound = (k * pieces + 2) * U32 * mag + 1e-30
    err = (got - ref).abs()
    assert (err <= bound).all(), float((err / bound).max())
