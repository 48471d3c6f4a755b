"""ksc_prox_g_batch (many vectors on device buffers, one CTA each) against the
FP64 oracle's prox (sort + PAVA merge, Alg. 1 + 4) row by row.  Both are exact up
to rounding: 1e-11 relative to the input scale, as for the single-vector prox."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


def _rows(count, p, seed, scale=1.0, tie=False):
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((count, p)) * scale
    if tie:
        w = np.round(w, 1)
    return w


def _check(K, w, k, M, rho, pad=0):
    import torch
    count, p = w.shape
    W = torch.zeros((count, p + pad), dtype=torch.float64, device="cuda")
    W[:, :p] = torch.from_numpy(w)
    out = torch.full((count, p + 2 * pad), 7.0, dtype=torch.float64, device="cuda")
    st = K.ksc_prox_g_batch(W.data_ptr(), W.stride(0), out.data_ptr(), out.stride(0), p, count, k, M, rho)
    assert st == K.KSC_OK, K.ksc_last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    tol = 1e-11 * max(1.0, np.abs(w).max())
    for r in range(count):
        ref, _ = O.prox_g(w[r], k, rho, M)
        assert np.max(np.abs(got[r, :p] - ref)) <= tol, (r, p, k)
    if pad:
        assert np.all(got[:, p:] == 7.0)   # nothing written past p in a padded row


@pytest.mark.parametrize("p,k", [(1, 1), (7, 3), (100, 10), (1000, 0), (1000, 1000), (4099, 10),
                                 (20011, 25), (12800, 10)])
def test_batch_rows_match_oracle(K, p, k):
    _check(K, _rows(5, p, seed=p + k), k, 1.0, 1.0)


@pytest.mark.parametrize("seed", range(6))
def test_batch_random_parameters_ties_and_padding(K, seed):
    rng = np.random.default_rng(100 + seed)
    p = int(rng.choice([31, 257, 3001, 9000]))
    k = int(rng.integers(0, 80))
    M = float(10 ** rng.uniform(-1, 1))
    rho = float(10 ** rng.uniform(-2, 3))
    _check(K, _rows(4, p, seed, scale=float(10 ** rng.uniform(-2, 1)), tie=seed % 2 == 0), k, M, rho, pad=3)


def test_batch_wide_pooled_block(K):
    # nearly equal magnitudes with rho = M = 10: ~6300 nonzeros per row, past the
    # 2048 candidates of a row's CTA -> the full-pass root
    rng = np.random.default_rng(7)
    w = rng.uniform(0.95, 1.0, (3, 20000)) * np.where(rng.random((3, 20000)) < 0.5, -1, 1)
    _check(K, w, 5, 10.0, 10.0)


def test_batch_equals_single_vector_prox(K):
    import torch
    w = _rows(6, 3000, seed=11)
    W = torch.from_numpy(w).cuda()
    out = K.prox_g_rows(W, 12, 1.5, 3.0)
    torch.cuda.synchronize()
    for r in range(6):
        single, _ = K.ksc_prox_g(w[r], 12, 1.5, 3.0)
        assert np.max(np.abs(out[r].cpu().numpy() - single)) <= 1e-12 * max(1.0, np.abs(w).max())


# ---- ksc_g_value_batch: g (Algorithm 2) of many device rows against the oracle's
# Algorithm 2 row by row (1e-12 relative), +inf outside dom g

def _g_check(K, B, k, M):
    import torch
    count, p = B.shape
    Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    g = K.g_value_rows(Bd, k, M)
    torch.cuda.synchronize()
    got = g.cpu().numpy()
    for r in range(count):
        ref = O.g_value(B[r], k, M)
        if np.isinf(ref):
            assert np.isinf(got[r]) and got[r] > 0, (r, got[r])
        else:
            assert abs(got[r] - ref) <= 1e-12 * max(1.0, abs(ref)), (r, p, k, got[r], ref)


@pytest.mark.parametrize("p,k", [(1, 1), (50, 5), (1000, 10), (1000, 1000), (12800, 10), (20011, 25)])
def test_g_value_rows_match_oracle(K, p, k):
    rng = np.random.default_rng(p + 7 * k)
    M = 1.5
    rows = []
    for r in range(6):
        # prox outputs lie in dom g: sparse, pooled (many equal magnitudes) and mixed rows
        w = rng.standard_normal(p) * (0.1 if r % 2 else 3.0)
        b, _ = O.prox_g(w, k, float(10 ** rng.uniform(-1, 2)), M)
        rows.append(b)
    flat = np.full(p, min(M, k * M / p) * 0.999)          # max |b| <= ||b||_1 / k: g = ||b||_1^2 / 2k
    rows.append(flat)
    over = rows[0].copy()
    over[0] = 1.01 * M                                      # outside the box
    rows.append(over)
    if k < p:
        wide = np.full(p, M * 0.999)                        # outside the l1 budget kM
        rows.append(wide)
    _g_check(K, np.array(rows), k, M)


def test_g_value_rows_reject_bad_arguments(K):
    import torch
    B = torch.zeros((2, 10), dtype=torch.float64, device="cuda")
    g = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert K.ksc_g_value_batch(B.data_ptr(), 5, 10, 2, 3, 1.0, g.data_ptr()) == K.KSC_ERR_INVALID_ARG   # ldb < p
    assert K.ksc_g_value_batch(B.data_ptr(), 10, 10, 2, 3, 0.0, g.data_ptr()) == K.KSC_ERR_INVALID_ARG  # M <= 0
    assert K.ksc_g_value_batch(B.data_ptr(), 10, 10, -1, 3, 1.0, g.data_ptr()) == K.KSC_ERR_INVALID_ARG
    assert K.ksc_g_value_batch(B.data_ptr(), 10, 10, 0, 3, 1.0, g.data_ptr()) == K.KSC_OK              # no rows
