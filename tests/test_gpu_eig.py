"""Eigen-perspective relaxation (App. D.2) through the CUDA path against the FP64
oracle, and the certified shift it rests on.

* The shift: the library's lambda (Cholesky-certified bisection) never exceeds
  the oracle's lambda_min(X^T X) (a dense FP64 eigensolver on the represented
  matrix) and lies within 2e-3 of it; a shift above lambda_min is refused.
* Parity: both sides solve with the same shift, taken from the oracle's
  lambda_min and certified by the library (so no input of the oracle comes from
  the CUDA path), to the tolerances of the batched parity tests: objective and
  certified bound within 1e-6 relative of the oracle's values at a 1e-12 gap, the
  bound never above the oracle's primal value.
"""
import numpy as np
import pytest

import ksc_inputs as G
from oracle import oracle as O
from tests import _pins as P

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


@pytest.mark.parametrize("dt", [G.F64, G.F32, G.BF16, "fp8"])
def test_eig_shift_is_a_certified_lower_bound(K, dt):
    # the small least-squares configuration: n = 500, p = 100, Toeplitz 0.5
    P0 = G.make_problem(500, 100, r=0.5, seed=0, x_dtype=G.F32 if dt == "fp8" else dt)
    if dt == "fp8":
        bits, s = G.quantize_fp8(P0.X)
        X = G.fp8_values(bits).astype(np.float64) * s.astype(np.float64)
        prob = K.Problem(bits, P0.y, K.KSC_LOSS_LSQ, x_dtype=K.KSC_FP8, col_scale=s)
    else:
        X = P0.X64() if dt == G.BF16 else np.asarray(P0.X, dtype=np.float64)
        prob = K.Problem(P0.X, P0.y, K.KSC_LOSS_LSQ)
    ref = O.lambda_min(X)
    lam = prob.eig_lambda()
    assert ref > 0 and (1 - 2e-3) * ref <= lam <= ref
    assert prob.eig_lambda() == lam                       # cached


def test_eig_shift_is_zero_below_full_rank_and_refused_above_lambda_min(K):
    P0 = G.make_problem(80, 120, r=0.5, seed=1, x_dtype=G.F64)
    assert K.Problem(P0.X, P0.y).eig_lambda() == 0.0      # n < p
    P1 = G.make_problem(300, 60, r=0.7, seed=2, x_dtype=G.F64)
    ref = O.lambda_min(P1.X)
    prob = K.Problem(P1.X, P1.y)
    with pytest.raises(K.KscError):
        prob.set_eig_lambda(1.01 * ref)
    prob.set_eig_lambda(0.99 * ref)
    assert prob.eig_lambda() == 0.99 * ref


def test_eig_batched_matches_oracle(K):
    P1 = G.make_problem(600, 120, r=0.5, seed=31, loss=G.LSQ, k_true=5, x_dtype=G.BF16, lambda2=0.5,
                        M=2.0, k=5)
    X = P1.X64()
    lam = float(0.999 * O.lambda_min(X))
    prob = K.Problem(P1.X, P1.y, K.KSC_LOSS_LSQ)
    prob.set_eig_lambda(lam)
    sets = G.node_sets(P1.p, 10, seed=3, max_zero=20, max_one=3)
    mk = lambda z, o, fl: K.Node(P1.lambda2, P1.M, P1.k, fixed_zero=z, fixed_one=o, rel_gap_tol=1e-7,
                                 max_iter=50000, flags=fl)
    res = prob.solve_batch([mk(z, o, K.KSC_FLAG_EIG) for z, o in sets], want_z=True)
    plain = prob.solve_batch([mk(z, o, 0) for z, o in sets])
    assert all(r.status == "ok" and r.rel_gap <= 1e-7 for r in res)
    for b in (0, 4, 9):
        zero, one = sets[b]
        st = _state(P1.p, zero, one)
        ref = O.solve(X, P1.y, 0, P1.lambda2, P1.M, P1.k, state=st, tol=1e-12, max_iter=200000, eig=lam)
        r = res[b]
        assert ref.status == "converged"
        assert _rel(r.dual_bound, ref.dual) <= 1e-6 and _rel(r.primal, ref.primal) <= 1e-6, b
        assert r.dual_bound <= ref.primal
        assert np.all(r.beta[zero] == 0) and np.all(r.z[zero] == 0) and np.all(r.z[one] == 1)
        # the oracle's eigen bound at the GPU's iterate agrees with the certificate
        assert _rel(O.dual_bound(X, P1.y, 0, P1.lambda2, P1.M, P1.k, r.beta, state=st, eig=lam),
                    r.dual_bound) <= 1e-6
    # tighter than the perspective bound of the same nodes
    for r, q in zip(res, plain):
        assert r.dual_bound >= q.dual_bound - 1e-6 * abs(q.dual_bound)
    assert sum(r.dual_bound - q.dual_bound for r, q in zip(res, plain)) > 0


def test_eig_needs_least_squares(K):
    P1 = G.make_problem(300, 60, r=0.5, seed=4, loss=G.LOGISTIC, x_dtype=G.BF16)
    prob = K.Problem(P1.X, P1.y, K.KSC_LOSS_LOGISTIC)
    with pytest.raises(K.KscError):
        prob.solve_batch([K.Node(0.1, 2.0, 5, flags=K.KSC_FLAG_EIG)])
    with pytest.raises(K.KscError):
        prob.solve(K.Node(0.1, 2.0, 5, flags=K.KSC_FLAG_EIG))


@pytest.mark.parametrize("dt", [G.F64, G.F32, G.BF16, "fp8"])
def test_eig_single_node_matches_oracle(K, dt):
    # the single-node path with the eigen-perspective relaxation (App. D.2): the
    # shifted gradient in the gradient pass, -eig ||b||^2 in the objective, eig
    # ||gamma||^2 in the in-loop dual term and the eigen bound with its margins in
    # the FP64 certificate -- against the oracle on the stored (represented) matrix
    P1 = G.make_problem(500, 100, r=0.5, seed=37, loss=G.LSQ, k_true=5, x_dtype=G.F32 if dt == "fp8" else dt,
                        lambda2=0.5, M=2.0, k=5)
    if dt == "fp8":
        bits, sc = G.quantize_fp8(P1.X)
        X = G.fp8_values(bits).astype(np.float64) * sc.astype(np.float64)
        prob = K.Problem(bits, P1.y, K.KSC_LOSS_LSQ, x_dtype=K.KSC_FP8, col_scale=sc)
    else:
        X = P1.X64() if dt == G.BF16 else np.asarray(P1.X, dtype=np.float64)
        prob = K.Problem(P1.X, P1.y, K.KSC_LOSS_LSQ)
    lam = float(0.999 * O.lambda_min(X))
    assert lam > 0
    prob.set_eig_lambda(lam)
    zero, one = np.array([3, 17, 40], np.int32), np.array([8], np.int32)
    st = _state(P1.p, zero, one)
    node = K.Node(P1.lambda2, P1.M, P1.k, fixed_zero=zero, fixed_one=one, rel_gap_tol=1e-8, max_iter=50000,
                  flags=K.KSC_FLAG_EIG)
    r = prob.solve(node)
    ref = O.solve(X, P1.y, 0, P1.lambda2, P1.M, P1.k, state=st, tol=1e-12, max_iter=200000, eig=lam)
    assert r.status == "ok" and r.rel_gap <= 1e-8
    assert ref.status == "converged"
    assert _rel(r.dual_bound, ref.dual) <= 1e-6 and _rel(r.primal, ref.primal) <= 1e-6
    assert r.dual_bound <= ref.primal
    assert np.all(r.beta[zero] == 0) and np.all(r.z[zero] == 0) and np.all(r.z[one] == 1)
    # the oracle's eigen bound at the GPU's iterate agrees with the certificate, which
    # stays below it (its margins)
    d_o = O.dual_bound(X, P1.y, 0, P1.lambda2, P1.M, P1.k, r.beta, state=st, eig=lam)
    assert r.dual_bound <= d_o + 1e-12 * abs(d_o) and _rel(r.dual_bound, d_o) <= 1e-8
    # tighter than the perspective bound of the same node
    plain = prob.solve(K.Node(P1.lambda2, P1.M, P1.k, fixed_zero=zero, fixed_one=one, rel_gap_tol=1e-8,
                              max_iter=50000))
    assert r.dual_bound > plain.dual_bound
    if dt == G.BF16:   # the batched path on the same node agrees
        rb = prob.solve_batch([node])[0]
        assert _rel(rb.dual_bound, r.dual_bound) <= 1e-6 and _rel(rb.primal, r.primal) <= 1e-6


def test_bnb_with_eig_node_bounds(K):
    Pm = G.make_problem(200, 14, r=0.9, seed=2, loss=G.LSQ, k_true=3, snr=3.0, x_dtype=G.BF16,
                        lambda2=0.1, M=2.0, k=4)
    X = Pm.X64()
    opt = P.mip_enumerate(X, Pm.y, 0.1, 2.0, 4, 0)
    prob = K.Problem(Pm.X, Pm.y, K.KSC_LOSS_LSQ, x_dtype=K.KSC_BF16)
    _, r0 = prob.bnb(0.1, 2.0, 4, opt_gap=1e-5, batch=64, node_rel_gap=1e-7, node_max_iter=30000)
    beta, r1 = prob.bnb(0.1, 2.0, 4, opt_gap=1e-5, batch=64, node_rel_gap=1e-7, node_max_iter=30000,
                        node_flags=K.KSC_FLAG_EIG)
    assert r0["certified"] and r1["certified"], (r0, r1)
    assert r1["lower_bound"] <= opt + 1e-9 * abs(opt)
    assert opt - 1e-9 * abs(opt) <= r1["incumbent"] <= opt + 2e-5 * abs(opt)
    assert np.count_nonzero(beta) <= 4 and np.abs(beta).max() <= 2.0
    assert r1["nodes"] <= 1.1 * r0["nodes"] + 8
