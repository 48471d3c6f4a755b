"""FP8 e4m3 X with power-of-two column scales (KSC_FP8_E4M3_COLSCALE) through the
single-node solver, against the FP64 oracle on the represented matrix
X~ = e4m3(bits) * s (exact in FP32, so the kernels' error-free products stay
exact with respect to X~).  Tolerances as for FP32/BF16 X: objective and
certified bound within 1e-6 relative of the oracle, beta (or u = X~ beta where beta
is not unique) within 1e-4 of its max-norm, and the bound never above the
oracle's primal value."""
import numpy as np
import pytest

import ksc_inputs as G
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


def _fp8(P):
    bits, s = G.quantize_fp8(P.X)
    Xt = G.fp8_values(bits).astype(np.float64) * s.astype(np.float64)
    return bits, s, Xt


@pytest.mark.parametrize("loss,n,p,seed", [(G.LSQ, 600, 300, 31), (G.LOGISTIC, 800, 257, 32),
                                           (G.LSQ, 300, 700, 33)])
def test_fp8_single_node_matches_oracle(K, loss, n, p, seed):
    P = G.make_problem(n, p, r=0.5, seed=seed, loss=loss, k_true=6, x_dtype=G.F32, lambda2=0.1, M=2.0, k=6)
    bits, s, Xt = _fp8(P)
    assert np.all(np.frexp(s)[0] == 0.5)          # powers of two
    prob = K.Problem(bits, P.y, K.KSC_LOSS_LSQ if loss == G.LSQ else K.KSC_LOSS_LOGISTIC,
                     x_dtype=K.KSC_FP8, col_scale=s)
    r = prob.solve(K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-7, max_iter=100000))
    ref = O.solve(Xt, P.y, loss, P.lambda2, P.M, P.k, tol=1e-12, max_iter=400000)
    assert r.status == "ok"
    assert _rel(r.dual_bound, ref.dual) <= 1e-6 and _rel(r.primal, ref.primal) <= 1e-6
    assert r.dual_bound <= ref.primal
    u, ur = Xt @ r.beta, Xt @ ref.beta
    assert np.max(np.abs(u - ur)) <= 1e-4 * max(1.0, np.abs(ur).max())
    # the problem's Lipschitz constant is that of X~
    lam, _ = O.power_iteration(Xt, tol=1e-13)
    c = 2.0 if loss == G.LSQ else 0.25
    theta = prob.L / (c * 1.01)   # the Lanczos Ritz value: within ~1e-3 below lambda_max
    assert lam * (1 - 2e-3) <= theta <= lam * (1 + 1e-9)


def test_fp8_node_with_fixed_sets_and_device_matrix(K):
    import torch
    P = G.make_problem(500, 200, r=0.7, seed=34, loss=G.LSQ, k_true=5, x_dtype=G.F32, lambda2=0.3, M=1.5, k=6)
    bits, s, Xt = _fp8(P)
    zero, one = np.array([3, 17, 40], np.int32), np.array([5, 90], np.int32)
    st = np.zeros(P.p, np.int8)
    st[zero] = O.ZERO
    st[one] = O.ONE
    node = K.Node(P.lambda2, P.M, P.k, fixed_zero=zero, fixed_one=one, rel_gap_tol=1e-7, max_iter=100000)
    host = K.Problem(bits, P.y, K.KSC_LOSS_LSQ, x_dtype=K.KSC_FP8, col_scale=s).solve(node)
    Xd = torch.from_numpy(bits).cuda().view(torch.float8_e4m3fn)
    dev = K.Problem(Xd, P.y, K.KSC_LOSS_LSQ, col_scale=s).solve(node)
    ref = O.solve(Xt, P.y, G.LSQ, P.lambda2, P.M, P.k, state=st, tol=1e-12, max_iter=400000)
    for r in (host, dev):
        assert r.status == "ok"
        assert _rel(r.dual_bound, ref.dual) <= 1e-6 and r.dual_bound <= ref.primal
        assert np.max(np.abs(r.beta - ref.beta)) <= 1e-4 * max(1.0, np.abs(ref.beta).max())
        assert np.all(r.beta[zero] == 0.0)
    # the same arithmetic from host or device storage
    assert host.dual_bound == dev.dual_bound and np.array_equal(host.beta, dev.beta)


def test_fp8_batch_call_uses_the_single_node_solver(K):
    P = G.make_problem(300, 120, r=0.5, seed=35, loss=G.LOGISTIC, k_true=4, x_dtype=G.F32, lambda2=0.2, M=2.0, k=4)
    bits, s, Xt = _fp8(P)
    prob = K.Problem(bits, P.y, K.KSC_LOSS_LOGISTIC, x_dtype=K.KSC_FP8, col_scale=s)
    nodes = [K.Node(P.lambda2, P.M, P.k, fixed_zero=[j], rel_gap_tol=1e-6) for j in range(3)]
    res = prob.solve_batch(nodes)
    for j, r in enumerate(res):
        st = np.zeros(P.p, np.int8)
        st[j] = O.ZERO
        ref = O.solve(Xt, P.y, G.LOGISTIC, P.lambda2, P.M, P.k, state=st, tol=1e-12, max_iter=400000)
        assert _rel(r.dual_bound, ref.dual) <= 1e-6 and r.dual_bound <= ref.primal
