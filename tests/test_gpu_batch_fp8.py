"""The batched solver on FP8 e4m3 X with power-of-two column scales, against the
FP64 oracle on the represented matrix.

With E4M3 X the lock-step products run on the tensor cores as kind::f8f6f4:
four E4M3 pieces of each node's difference from its anchor (scaled per node by a
power of two; the forward pieces carry s_j (beta_j - beta_ref_j), the column
scales folded in) against the stored E4M3 X, the inverse scales and the column
scales applied in the epilogue.  The anchors and certificates use the exact
tensor-core product of the represented matrix X_ij s_j (exact in BF16).  The
problem solved is the represented matrix, so the oracle runs on it in FP64.

Cases: logistic with p not a multiple of 16 (the E4M3 rows are copied to a
16-byte stride), admitted as 8 nodes (each node's exact anchor at its warm start)
and as 40 (the zero anchor); least squares with p a multiple of 16 (X read in
place).  Compared with the oracle solved to a 1e-12 gap: certified bound and
objective within 1e-6 relative, beta within 1e-4 of its max-norm.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import ksc_inputs as G
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]


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


def _case(n, p, loss, seed, lambda2, M, k):
    P = G.make_problem(n, p, r=0.5, seed=seed, loss=loss, k_true=min(k, 10), x_dtype=G.F32,
                       lambda2=lambda2, M=M, k=k)
    bits, s = G.quantize_fp8(P.X)
    Xt = G.fp8_values(bits).astype(np.float64) * s.astype(np.float64)[None, :]
    root = O.solve(Xt, P.y, P.loss, lambda2, M, k, tol=1e-6, max_iter=200000)
    assert root.status == "converged"
    return P, bits, s, Xt, root


@pytest.mark.parametrize("loss,n,p,count,check", [
    (G.LOGISTIC, 600, 1500, 8, (0, 5)),
    (G.LOGISTIC, 600, 1500, 40, (1, 2)),
    (G.LSQ, 500, 1024, 8, (0, 4)),
])
def test_batched_fp8_matches_oracle_on_represented_matrix(K, loss, n, p, count, check):
    lambda2, M, k = (3.0, 3.0, 20) if loss == G.LOGISTIC else (1.0, 2.0, 10)
    P, bits, s, Xt, root = _case(n, p, loss, 51 + count, lambda2, M, k)
    sets = G.node_sets(p, count, seed=13, max_zero=100, max_one=min(9, k - 1))
    pert = G.warm_perturbation(p, count, seed=13)
    warms = [root.beta + pert[b] for b in range(count)]
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=len(check), mp_context=ctx) as pool:
        futs = {b: pool.submit(O.solve, Xt, P.y, P.loss, lambda2, M, k, state=_state(p, *sets[b]),
                               warm=warms[b], L=root.L, tol=1e-12, max_iter=60000)
                for b in check}
        prob = K.Problem(bits, P.y, loss, x_dtype=K.KSC_FP8, col_scale=s)
        nodes = [K.Node(lambda2, M, k, fixed_zero=sets[b][0], fixed_one=sets[b][1], warm_beta=warms[b],
                        rel_gap_tol=1e-7, max_iter=30000) for b in range(count)]
        res = prob.solve_batch(nodes, want_z=True)
        stats = K.ksc_problem_solve_stats(prob.h)
        refs = {b: f.result() for b, f in futs.items()}
    assert stats["batch_anchors"] > 0, stats      # the batched path ran
    assert all(r.status == "ok" and r.rel_gap <= 1e-7 for r in res), \
        [(b, r.status, r.iters, r.rel_gap) for b, r in enumerate(res)]
    for b in check:
        zero, one = sets[b]
        r, ref = res[b], refs[b]
        assert ref.status == "converged", (b, ref.status, ref.gap)
        assert _rel(r.dual_bound, ref.dual) <= 1e-6, (b, r.dual_bound, ref.dual)
        assert _rel(r.primal, ref.primal) <= 1e-6, (b, r.primal, ref.primal)
        assert r.dual_bound <= ref.primal
        scale = max(1.0, np.abs(ref.beta).max())
        assert np.max(np.abs(r.beta - ref.beta)) <= 1e-4 * scale, (b, np.max(np.abs(r.beta - ref.beta)))
        assert np.all(r.beta[zero] == 0) and np.all(r.z[one] == 1)
