"""The exact product of the batched solver's anchors and certificates on the
tensor cores (ksc_tc_exact), against a double-double reference.

The certificate of Sec. 3.4 is a valid bound only if X^T zeta is known to an
accuracy its margin covers.  The kernel splits BF16 X and the FP64 vectors into
8-bit fixed-point slices and sums every slice product exactly, so its result
must lie within its stated bound eps ||A_j|| ||V_i|| of the exact product, and in
practice within the vector's truncation below 2^-47 of its largest entry.  The reference splits each V entry
into two halves whose products with an 8-bit BF16 entry are exact in FP64 and
accumulates them with TwoSum (double-double), which is exact to ~K u^2.

Cases: K split over several CTAs (few tiles) and not split (>= 304 tiles); K not a
multiple of 64 (the TMA's zero fill); rows of A with entries below 2^-16 of
their largest (the sparse exact residual), a row with one outlier, a zero row;
vectors that are zero or scaled by 1e-30 and 1e30.
"""
import numpy as np
import pytest

import ksc_inputs as G

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


def _bf16(x):
    """Round to BF16 (nearest even) and return (bits as uint16, values as float64)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
    return r, G.bf16_to_f32(r).astype(np.float64)


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _exact(A, V, rs, cs):
    """sum_k A[c, k] V[r, k] for the pairs (rs[i], cs[i]) in double-double."""
    a, v = A[cs], V[rs]
    t = v * 134217729.0                      # Veltkamp split: 26 + 27 bits
    hi = t - (t - v)
    lo = v - hi
    p1, p2 = a * hi, a * lo                  # exact: 8-bit a times <= 27-bit halves
    s = np.zeros(len(rs))
    e = np.zeros(len(rs))
    for k in range(A.shape[1]):
        s, d = _two_sum(s, p1[:, k])
        e += d
        s, d = _two_sum(s, p2[:, k])
        e += d
    return s + e


def _case(C, Kd, R, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((C, Kd)).astype(np.float32)
    A[0] = 0.0                                        # zero row
    A[1, ::7] *= 1e-7                                 # entries far below the row's top: residuals
    A[2, 5] = 3.0e4                                   # one outlier: most of the row leaves residuals
    bits, A64 = _bf16(A)
    V = rng.standard_normal((R, Kd))
    V[0] = 0.0
    V[1] *= 1e-30
    if R > 2:
        V[2] *= 1e30
    V[R - 1, ::3] = 0.0
    return bits, A64, V


@pytest.mark.parametrize("C,Kd,R,sampled", [(700, 3000, 37, False), (333, 1000, 5, False),
                                            (2432, 512, 512, True)])
def test_exact_product_matches_double_double(K, C, Kd, R, sampled):
    import torch
    torch.cuda.set_device(0)
    bits, A64, V = _case(C, Kd, R, seed=C + Kd + R)
    Ad = torch.from_numpy(bits.view(np.int16)).cuda()
    Vd = torch.from_numpy(V).cuda()
    Dd = torch.full((R, C), float("nan"), dtype=torch.float64, device="cuda")
    eps = K.ksc_tc_exact(Ad.data_ptr(), C, Kd, Kd, Vd.data_ptr(), R, Kd, Dd.data_ptr(), C)
    D = Dd.cpu().numpy()
    assert np.all(np.isfinite(D))
    assert 0 < eps < 2e-12
    if sampled:
        rng = np.random.default_rng(7)
        rs = np.concatenate([np.arange(3), rng.integers(0, R, 3000)])
        cs = np.concatenate([np.arange(3), rng.integers(0, C, 3000)])
    else:
        rs, cs = np.meshgrid(np.arange(R), np.arange(C), indexing="ij")
        rs, cs = rs.ravel(), cs.ravel()
    ref = _exact(A64, V, rs, cs)
    got = D[rs, cs]
    err = np.abs(got - ref)
    # the stated rigorous bound
    bound = eps * np.linalg.norm(A64[cs], axis=1) * np.linalg.norm(V[rs], axis=1)
    assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
    # and in practice: the truncation of each vector below 2^-47 of its largest
    # entry (times ||A_j||_1), plus the last bits of sum |a v| -- far below the
    # ~1e-8 an inexact FP32 accumulation would leave
    mag = np.sum(np.abs(A64[cs] * V[rs]), axis=1)
    trunc = 2.0 ** -46 * np.sum(np.abs(A64[cs]), axis=1) * np.max(np.abs(V[rs]), axis=1)
    assert np.all(err <= trunc + 1e-14 * mag), float(np.max(err / np.maximum(trunc + mag, 1e-300)))
    # zero row / zero vector give exact zeros
    assert np.all(D[0] == 0.0) and np.all(D[:, 0] == 0.0)
