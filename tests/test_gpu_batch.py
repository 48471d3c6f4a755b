"""Batched solves (ksc_solve_batch: tensor-core products, one prox CTA per node)
against the FP64 oracle, on the same seeded inputs.

The batched path keeps the iterate in FP64 and multiplies BF16 X by differences
from per-node anchors on the tensor cores (three BF16 pieces whose sum is the FP32
difference exactly; FP32 accumulation), and every reported bound is the FP64
certificate at the final iterate.  The tolerances are the ones of the single-node
FP32/BF16 path: objective and certified bound within
1e-6 relative of the oracle's values at a 1e-12 gap, the bound never above the
oracle's primal value, beta within 1e-4 relative to its max-norm where the
solution is unique (n > p, strictly convex loss).

Warm starts are the oracle's own root solution plus a seeded N(0, 1e-2)
perturbation, so no input of the oracle comes from the CUDA path.
"""
import math

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


def _nodes(K, P, count, seed, warm_root, max_zero, max_one, tol=1e-7):
    sets = G.node_sets(P.p, count, seed=seed, max_zero=max_zero, max_one=max_one)
    pert = G.warm_perturbation(P.p, count, seed=seed)
    out = []
    for b, (zero, one) in enumerate(sets):
        warm = warm_root + pert[b] if warm_root is not None else None
        out.append((zero, one, warm,
                    K.Node(P.lambda2, P.M, P.k, fixed_zero=zero, fixed_one=one, warm_beta=warm,
                           rel_gap_tol=tol, max_iter=30000)))
    return out


@pytest.fixture(scope="module")
def logistic_case():
    # logistic, BF16 X, p*2 bytes not a multiple of 16 (the TMA path copies X)
    P = G.make_problem(800, 300, r=0.5, seed=21, loss=G.LOGISTIC, k_true=10, x_dtype=G.BF16,
                       lambda2=0.05, M=3.0, k=10)
    root = O.solve(_X(P), P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-9, max_iter=200000)
    return P, root


def test_batched_logistic_bf16_matches_oracle(K, logistic_case):
    P, root = logistic_case
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_LOGISTIC)
    nodes = _nodes(K, P, 12, seed=5, warm_root=root.beta, max_zero=40, max_one=5)
    res = prob.solve_batch([n[3] for n in nodes], want_z=True)
    for b in range(0, 12, 2):
        zero, one, warm, _ = nodes[b]
        r = res[b]
        st = _state(P.p, zero, one)
        ref = O.solve(_X(P), P.y, P.loss, P.lambda2, P.M, P.k, state=st, warm=warm, tol=1e-12,
                      max_iter=200000)
        assert r.status == "ok" and r.rel_gap <= 1e-7, (b, r)
        assert _rel(r.dual_bound, ref.dual) <= 1e-6 and _rel(r.primal, ref.primal) <= 1e-6, b
        assert r.dual_bound <= ref.primal
        assert np.max(np.abs(r.beta - ref.beta)) <= 1e-4 * max(1.0, np.abs(ref.beta).max())
        assert np.all(r.beta[zero] == 0) and np.all(r.z[zero] == 0) and np.all(r.z[one] == 1)
    # every node of the batch is certified
    assert all(r.status == "ok" and r.rel_gap <= 1e-7 for r in res)


def test_batched_matches_single_node_and_is_order_invariant(K, logistic_case):
    P, root = logistic_case
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_LOGISTIC)
    nodes = _nodes(K, P, 9, seed=8, warm_root=root.beta, max_zero=40, max_one=5)
    res = prob.solve_batch([n[3] for n in nodes])
    # the same node alone and at another position of a different batch
    alone = prob.solve_batch([nodes[4][3]])[0]
    mixed = prob.solve_batch([nodes[i][3] for i in (7, 4, 1)])[1]
    single = prob.solve(nodes[4][3])
    for other in (alone, mixed, single):
        assert _rel(other.dual_bound, res[4].dual_bound) <= 1e-6
        assert _rel(other.primal, res[4].primal) <= 1e-6
    # alone and in the mix the node follows the same arithmetic up to the summation
    # order of its exact products (split over more CTAs when few nodes share them)
    for other in (alone, mixed):
        assert _rel(other.dual_bound, res[4].dual_bound) <= 1e-6
        assert np.max(np.abs(other.beta - res[4].beta)) <= 1e-4 * max(1.0, np.abs(res[4].beta).max())


def test_batched_lsq_ragged_batch_with_special_nodes(K):
    # least squares, BF16 X, 130 nodes (a ragged second tile of 128 node rows)
    P = G.make_problem(600, 256, r=0.7, seed=23, loss=G.LSQ, k_true=6, x_dtype=G.BF16,
                       lambda2=0.3, M=2.0, k=6)
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_LSQ)
    nodes = _nodes(K, P, 130, seed=9, warm_root=None, max_zero=30, max_one=3)
    ns = [n[3] for n in nodes]
    # node 3: k' = 0 (S1 has k elements); node 7: infeasible (S0 and S1 intersect)
    one3 = np.arange(P.k, dtype=np.int32)
    ns[3] = K.Node(P.lambda2, P.M, P.k, fixed_one=one3, rel_gap_tol=1e-7)
    ns[7] = K.Node(P.lambda2, P.M, P.k, fixed_zero=[5, 6], fixed_one=[6], rel_gap_tol=1e-7)
    res = prob.solve_batch(ns, want_z=True)
    assert res[7].status == "infeasible_node" and res[7].dual_bound == math.inf and res[7].pruned
    for b in (0, 3, 64, 127, 128, 129):
        if b == 3:
            zero, one = np.zeros(0, np.int32), one3
        else:
            zero, one = nodes[b][0], nodes[b][1]
        st = _state(P.p, zero, one)
        ref = O.solve(_X(P), P.y, P.loss, P.lambda2, P.M, P.k, state=st, tol=1e-12, max_iter=200000)
        r = res[b]
        assert r.status == "ok" and r.rel_gap <= 1e-7, (b, r)
        assert _rel(r.dual_bound, ref.dual) <= 1e-6 and _rel(r.primal, ref.primal) <= 1e-6, b
        assert r.dual_bound <= ref.primal
        assert np.max(np.abs(r.beta - ref.beta)) <= 1e-4 * max(1.0, np.abs(ref.beta).max())
    # k' = 0: the free coordinates are zero
    free3 = np.ones(P.p, bool)
    free3[one3] = False
    assert np.all(res[3].beta[free3] == 0)


def test_batched_incumbent_prunes_and_branches(K):
    P = G.make_problem(500, 200, r=0.5, seed=24, loss=G.LSQ, k_true=5, x_dtype=G.BF16,
                       lambda2=0.5, M=2.0, k=5)
    prob = K.Problem(P.X, P.y, K.KSC_LOSS_LSQ)
    ref = O.solve(_X(P), P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-12, max_iter=200000)
    low = K.Node(P.lambda2, P.M, P.k, incumbent=0.5 * ref.dual, rel_gap_tol=1e-9)
    high = K.Node(P.lambda2, P.M, P.k, incumbent=2.0 * ref.primal, rel_gap_tol=1e-9)
    plain = K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-9)
    r_low, r_high, r_plain = prob.solve_batch([low, high, plain])
    # incumbent below the bound: pruned with a certified bound above it
    assert r_low.pruned and r_low.dual_bound > 0.5 * ref.dual
    # incumbent far above: the primal drops below it (branch rule), bound valid
    assert not r_high.pruned and r_high.dual_bound <= ref.primal
    assert r_plain.status == "ok" and _rel(r_plain.dual_bound, ref.dual) <= 1e-6


def test_batch_on_fp32_x_runs_the_single_node_solver(K):
    P = G.make_problem(300, 90, r=0.5, seed=25, loss=G.LSQ, k_true=4, x_dtype=G.F32,
                       lambda2=0.5, M=2.0, k=4)
    prob = K.Problem(P.X, P.y)
    nodes = _nodes(K, P, 3, seed=3, warm_root=None, max_zero=10, max_one=2)
    res = prob.solve_batch([n[3] for n in nodes])
    for (zero, one, warm, nd), r in zip(nodes, res):
        s = prob.solve(nd)
        assert r.dual_bound == s.dual_bound and np.array_equal(r.beta, s.beta)
