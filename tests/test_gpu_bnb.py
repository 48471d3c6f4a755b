"""Branch and bound (ksc_bnb_solve) against the exact optimum of Eq. (1) found by
enumerating every support (each solved as a box-constrained ridge problem), on
small BF16 problems.  The oracle side runs on the stored matrix promoted to FP64.

Tolerances: the incumbent is the FP64 objective of a feasible point, so it can
not lie below the optimum (beyond rounding, 1e-9) and must reach it within the
certification tolerance; the lower bound is certified, so it never exceeds the
optimum; the returned point satisfies |b| <= M, ||b||_0 <= k and reproduces the
incumbent value."""
import numpy as np
import pytest

import ksc_inputs as G
from tests import _pins as P

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


def _objective(X, y, loss, lam, b):
    u = X @ b
    if loss == G.LSQ:
        f = np.sum((u - y) ** 2)
    elif loss == G.SQHINGE:
        f = np.sum(np.maximum(0.0, 1.0 - y * u) ** 2)
    else:
        f = np.sum(np.logaddexp(0.0, -y * u))
    return float(f + lam * b @ b)


CASES = [  # loss, n, p, k, lambda2, M, r, seed
    (G.LSQ, 120, 12, 3, 0.5, 1.5, 0.5, 1),
    (G.LSQ, 200, 14, 4, 0.1, 2.0, 0.9, 2),
    (G.LOGISTIC, 160, 11, 3, 0.2, 2.0, 0.5, 3),
    (G.LOGISTIC, 240, 12, 2, 0.05, 3.0, 0.1, 4),
    (G.SQHINGE, 160, 11, 3, 0.2, 2.0, 0.5, 5),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{['ls', 'logit', 'sqhinge'][c[0]]}_p{c[2]}_k{c[3]}")
def test_bnb_certifies_the_enumerated_optimum(K, case):
    loss, n, p, k, lam, M, r, seed = case
    Pm = G.make_problem(n, p, r=r, seed=seed, loss=loss, k_true=min(k, 3), snr=3.0, x_dtype=G.BF16,
                        lambda2=lam, M=M, k=k)
    X = Pm.X64()
    opt = P.mip_enumerate(X, Pm.y, lam, M, k, loss)
    prob = K.Problem(Pm.X, Pm.y, loss, x_dtype=K.KSC_BF16)
    beta, res = prob.bnb(lam, M, k, opt_gap=1e-5, batch=64, node_rel_gap=1e-7, node_max_iter=30000)
    assert res["certified"], res
    assert res["lower_bound"] <= opt + 1e-9 * abs(opt)
    assert res["incumbent"] >= opt - 1e-9 * abs(opt)
    assert res["incumbent"] <= opt + 2e-5 * abs(opt)
    assert res["gap"] <= 1e-5
    assert np.count_nonzero(beta) <= k and np.abs(beta).max() <= M
    assert abs(_objective(X, Pm.y, loss, lam, beta) - res["incumbent"]) <= 1e-9 * abs(opt)
    assert res["nodes"] >= 1 and res["heuristic_solves"] >= 1


def test_bnb_node_budget_leaves_a_valid_bound(K):
    loss, n, p, k, lam, M, r, seed = (G.LSQ, 200, 14, 4, 0.1, 2.0, 0.9, 2)
    Pm = G.make_problem(n, p, r=r, seed=seed, loss=loss, k_true=3, snr=3.0, x_dtype=G.BF16,
                        lambda2=lam, M=M, k=k)
    opt = P.mip_enumerate(Pm.X64(), Pm.y, lam, M, k, loss)
    prob = K.Problem(Pm.X, Pm.y, K.KSC_LOSS_LSQ, x_dtype=K.KSC_BF16)
    beta, res = prob.bnb(lam, M, k, opt_gap=0.0, max_nodes=3, batch=2)
    assert res["nodes"] <= 3 + 2         # nodes already in flight when the budget is reached finish
    assert res["lower_bound"] <= opt + 1e-9 * abs(opt)
    assert res["incumbent"] >= opt - 1e-9 * abs(opt)


def test_bnb_needs_bf16(K):
    Pm = G.cfg_small_lsq(seed=0)
    prob = K.Problem(Pm.X, Pm.y, K.KSC_LOSS_LSQ)
    with pytest.raises(K.KscError):
        prob.bnb(Pm.lambda2, Pm.M, Pm.k)
