"""Squared-hinge loss (App. D.1) through the CUDA path against the FP64 oracle.

The tolerances are those of the least-squares and logistic parity tests:
objective and certified bound within 1e-6 relative of the oracle's values at a
1e-12 gap, the bound never above the oracle's primal value.  The squared hinge
is flat where a margin is met, so the minimiser need not be unique: beta is
compared through the objective, the bound and feasibility (|S| <= k is not
required of the relaxation, |beta| <= M and the fixed sets are).

Warm starts of the batched nodes are the oracle's own root solution plus a seeded
N(0, 1e-2) perturbation, so no input of the oracle comes from the CUDA path.
"""
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


def _X(P):
    return P.X64() if P.x_dtype == G.BF16 else P.X


def _state(p, zero, one):
    st = np.zeros(p, np.int8)
    st[zero] = O.ZERO
    st[one] = O.ONE
    return st


def _check(r, ref, M, zero=(), one=()):
    assert r.status == "ok", r
    assert _rel(r.dual_bound, ref.dual) <= 1e-6 and _rel(r.primal, ref.primal) <= 1e-6
    assert r.dual_bound <= ref.primal
    assert r.dual_bound <= r.primal
    assert np.abs(r.beta).max() <= M
    assert np.all(r.beta[np.asarray(zero, dtype=np.int64)] == 0)


@pytest.mark.parametrize("seed", [1, 2])
def test_sqhinge_f64_matches_oracle(K, seed):
    P = G.make_problem(400, 90, r=0.5, seed=seed, loss=G.SQHINGE, k_true=5, x_dtype=G.F64,
                       lambda2=0.5, M=2.0, k=5)
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_SQHINGE)
    r = prob.solve(K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-10, max_iter=50000))
    ref = O.solve(P.X, P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-12, max_iter=200000)
    assert ref.status == "converged"
    _check(r, ref, P.M)
    assert r.rel_gap <= 1e-10
    # the oracle's objective at the GPU's beta agrees with the GPU's own value
    assert _rel(O.primal(P.X, P.y, P.loss, P.lambda2, P.M, P.k, r.beta), r.primal) <= 1e-9


def test_sqhinge_f32_node_with_fixed_sets(K):
    P = G.make_problem(500, 200, r=0.7, seed=3, loss=G.SQHINGE, k_true=6, x_dtype=G.F32,
                       lambda2=0.2, M=1.5, k=6)
    nz = np.nonzero(P.beta_star)[0]
    zero = np.array(sorted({int(nz[0]), 3, 11, 40}), np.int32)
    one = np.array([int(nz[1]), 150], np.int32)
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_SQHINGE)
    r = prob.solve(K.Node(P.lambda2, P.M, P.k, fixed_zero=zero, fixed_one=one, rel_gap_tol=1e-8,
                          max_iter=100000), want_z=True)
    ref = O.solve(P.X, P.y, P.loss, P.lambda2, P.M, P.k, state=_state(P.p, zero, one), tol=1e-12,
                  max_iter=200000)
    _check(r, ref, P.M, zero, one)
    assert np.all(r.z[zero] == 0) and np.all(r.z[one] == 1)


def test_sqhinge_batched_bf16_matches_oracle(K):
    P = G.make_problem(800, 300, r=0.5, seed=21, loss=G.SQHINGE, k_true=10, x_dtype=G.BF16,
                       lambda2=0.05, M=3.0, k=10)
    root = O.solve(_X(P), P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-9, max_iter=200000)
    sets = G.node_sets(P.p, 10, seed=5, max_zero=40, max_one=5)
    pert = G.warm_perturbation(P.p, 10, seed=5)
    nodes = [K.Node(P.lambda2, P.M, P.k, fixed_zero=z, fixed_one=o, warm_beta=root.beta + pert[b],
                    rel_gap_tol=1e-7, max_iter=30000) for b, (z, o) in enumerate(sets)]
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_SQHINGE)
    res = prob.solve_batch(nodes)
    assert all(r.status == "ok" and r.rel_gap <= 1e-7 for r in res)
    for b in (0, 3, 9):
        zero, one = sets[b]
        ref = O.solve(_X(P), P.y, P.loss, P.lambda2, P.M, P.k, state=_state(P.p, zero, one),
                      warm=root.beta + pert[b], tol=1e-12, max_iter=200000)
        _check(res[b], ref, P.M, zero, one)
    # the same node alone on the single-node path
    single = prob.solve(nodes[3])
    assert _rel(single.dual_bound, res[3].dual_bound) <= 1e-6


def test_sqhinge_zero_anchor_batch(K):
    # 40 cold-started nodes: the batch takes the zero anchor (u_ref = 0,
    # r_ref = grad F(0) = -2 y for the squared hinge)
    P = G.make_problem(600, 256, r=0.5, seed=24, loss=G.SQHINGE, k_true=6, x_dtype=G.BF16,
                       lambda2=0.1, M=2.0, k=6)
    sets = G.node_sets(P.p, 40, seed=11, max_zero=30, max_one=3)
    nodes = [K.Node(P.lambda2, P.M, P.k, fixed_zero=z, fixed_one=o, rel_gap_tol=1e-7, max_iter=30000)
             for z, o in sets]
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_SQHINGE)
    res = prob.solve_batch(nodes)
    assert all(r.status == "ok" and r.rel_gap <= 1e-7 for r in res)
    for b in (0, 21, 39):
        zero, one = sets[b]
        ref = O.solve(_X(P), P.y, P.loss, P.lambda2, P.M, P.k, state=_state(P.p, zero, one),
                      tol=1e-12, max_iter=200000)
        _check(res[b], ref, P.M, zero, one)
