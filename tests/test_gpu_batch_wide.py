"""The batched path as the batched benchmark runs it, against the FP64 oracle.

The batched workload (logistic loss, BF16 X, hundreds of warm-started nodes with
fixed sets as in App. B.3) takes two routes that small batches never reach:

* admissions of 32 or more nodes start from the zero anchor (beta_ref = 0,
  r_ref = grad F(0) in closed form, one shared G_ref = X^T grad F(0)), so the first
  products of every node are differences from 0, not from its own warm start;
* warm starts perturbed by N(0, 1e-2) make every coordinate nonzero, and the
  pooled tail of the prox of Alg. 1 + Alg. 4 (the coordinates above the threshold
  outside the top k') then exceeds the 2048 candidates a node keeps in shared
  memory, so the prox takes its full-pass root search, warm-started at the
  previous step's threshold.

This module solves 40 such nodes of a 600 x 4096 logistic problem in one batch
and compares the four with the largest budgets k' (the widest pooled tails)
element by element with the oracle solved to a 1e-12 gap: certified bound and
objective within 1e-6 relative, the bound never above the oracle's objective,
beta within 1e-4 of its max-norm (lambda2 = 3 makes the node problems strongly
convex, so beta is unique).  lambda2 = 3 keeps the oracle's solves to about a
minute each; the pooled tails still pass 2048 on the first steps (about 2100 to
2700 coordinates by the oracle's own iteration).  The oracle's solves run in
spawned worker processes while the GPU works.

Warm starts are the oracle's root solution plus a seeded perturbation, so no
input of the oracle comes from the CUDA path.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

import ksc_inputs as G
from oracle import oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]

N_NODES = 40      # >= 32: the zero-anchor admission
N_CHECK = 4       # nodes compared with the oracle element by element


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


@pytest.fixture(scope="module")
def wide_case():
    P = G.make_problem(600, 4096, r=0.5, seed=31, loss=G.LOGISTIC, k_true=10, x_dtype=G.BF16,
                       lambda2=3.0, M=3.0, k=20)
    X = P.X64()
    root = O.solve(X, P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-6, max_iter=200000)
    assert root.status == "converged"
    sets = G.node_sets(P.p, N_NODES, seed=7, max_zero=200, max_one=9)
    pert = G.warm_perturbation(P.p, N_NODES, seed=7)
    warms = [root.beta + pert[b] for b in range(N_NODES)]
    # the widest budgets k' = k - |S1| (ties by node index)
    check = sorted(range(N_NODES), key=lambda b: (len(sets[b][1]), b))[:N_CHECK]
    return P, X, root, sets, warms, check


def test_batched_wide_logistic_matches_oracle(K, wide_case):
    P, X, root, sets, warms, check = wide_case
    # the oracle's node solves start first, in spawned processes (never forked
    # from a process that holds a CUDA context), and run while the GPU works
    ctx = mp.get_context("spawn")
    workers = max(1, min(N_CHECK, os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as pool:
        futs = {b: pool.submit(O.solve, X, P.y, P.loss, P.lambda2, P.M, P.k,
                               state=_state(P.p, *sets[b]), warm=warms[b], L=root.L,
                               tol=1e-12, max_iter=60000)
                for b in check}
        prob = K.Problem(P.X, P.y, K.KSC_LOSS_LOGISTIC)
        nodes = [K.Node(P.lambda2, P.M, P.k, fixed_zero=sets[b][0], fixed_one=sets[b][1],
                        warm_beta=warms[b], rel_gap_tol=1e-7, max_iter=30000)
                 for b in range(N_NODES)]
        res = prob.solve_batch(nodes, want_z=True)
        stats = K.ksc_problem_solve_stats(prob.h)
        # one of the compared nodes again, alone (a one-node admission: its own exact
        # anchor instead of the zero anchor)
        alone = prob.solve_batch([nodes[check[0]]])[0]
        refs = {b: f.result() for b, f in futs.items()}

    # the full-pass root search of the prox ran (pooled tails past the candidates)
    assert stats["prox_fallback"] > 0, stats
    assert all(r.status == "ok" and r.rel_gap <= 1e-7 for r in res), \
        [(b, r.status, r.rel_gap) for b, r in enumerate(res) if r.status != "ok" or r.rel_gap > 1e-7]
    for b in check:
        zero, one = sets[b]
        r, ref = res[b], refs[b]
        assert ref.status == "converged", (b, ref.status, ref.gap)
        assert _rel(r.dual_bound, ref.dual) <= 1e-6, (b, r.dual_bound, ref.dual)
        assert _rel(r.primal, ref.primal) <= 1e-6, (b, r.primal, ref.primal)
        assert r.dual_bound <= ref.primal, (b, r.dual_bound, ref.primal)
        scale = max(1.0, np.abs(ref.beta).max())
        assert np.max(np.abs(r.beta - ref.beta)) <= 1e-4 * scale, (b, np.max(np.abs(r.beta - ref.beta)))
        assert np.all(r.beta[zero] == 0) and np.all(r.z[zero] == 0) and np.all(r.z[one] == 1)
        assert np.abs(r.beta).max() <= P.M
    # the same node alone and in the batch
    b0 = check[0]
    assert alone.status == "ok"
    assert _rel(alone.dual_bound, res[b0].dual_bound) <= 1e-6
    assert _rel(alone.primal, res[b0].primal) <= 1e-6
    assert np.max(np.abs(alone.beta - res[b0].beta)) <= 1e-4 * max(1.0, np.abs(res[b0].beta).max())
