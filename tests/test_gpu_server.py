"""The serving loop (ksc_server_*): continuous batching of node solves over
resident problems, admission by HBM budget, and results that are the same alone
and in the mix.

Each served result is checked against the same node solved alone by
ksc_solve_batch (a batch of one): certified bound and primal value within the
1e-6 relative tolerance of the batched path, gap at or below the node's target.
"""
import time

import numpy as np
import pytest

import ksc_inputs as G

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(400)]


@pytest.fixture(scope="module")
def K():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc
    return ksc


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


@pytest.fixture(scope="module")
def problems(K):
    P1 = G.make_problem(900, 400, r=0.5, seed=31, loss=G.LOGISTIC, k_true=8, x_dtype=G.BF16,
                        lambda2=0.05, M=3.0, k=8)
    P2 = G.make_problem(700, 320, r=0.9, seed=32, loss=G.LSQ, k_true=6, x_dtype=G.BF16,
                        lambda2=0.1, M=2.0, k=6)
    pr1 = K.Problem(P1.X, P1.y, K.KSC_LOSS_LOGISTIC)
    pr2 = K.Problem(P2.X, P2.y, K.KSC_LOSS_LSQ)
    return (P1, pr1), (P2, pr2)


def _nodes(K, P, count, seed, tol=1e-7):
    sets = G.node_sets(P.p, count, seed=seed, max_zero=30, max_one=3)
    return [K.Node(P.lambda2, P.M, P.k, fixed_zero=z, fixed_one=o, rel_gap_tol=tol, max_iter=30000)
            for z, o in sets]


def test_served_results_match_the_node_alone(K, problems):
    (P1, pr1), (P2, pr2) = problems
    n1, n2 = _nodes(K, P1, 10, seed=1), _nodes(K, P2, 10, seed=2)
    sv = K.Server(hbm_budget_bytes=8 << 30, max_slots=8)
    try:
        tickets = []
        for a, b in zip(n1, n2):   # interleaved arrivals of two problems
            tickets.append((pr1, a, sv.submit(pr1, a)))
            tickets.append((pr2, b, sv.submit(pr2, b)))
        served = [(pr, nd, sv.poll(t, timeout_ms=120000)) for pr, nd, t in tickets]
        st = sv.stats()
    finally:
        sv.close()
    assert st["completed"] == 20 and st["sessions"] >= 2
    # 10 nodes per problem on 8 slots: the last two are admitted while others run
    assert st["admitted_while_running"] >= 2
    for pr, nd, r in served:
        assert r is not None and r.status == "ok" and r.rel_gap <= 1e-7
        alone = pr.solve_batch([nd])[0]
        assert _rel(r.dual_bound, alone.dual_bound) <= 1e-6
        assert _rel(r.primal, alone.primal) <= 1e-6


def test_admission_by_budget(K, problems):
    (P1, pr1), (P2, pr2) = problems
    # a budget that holds one problem's session at a time: the second problem waits
    one = max(pr1.bytes, pr2.bytes) * 2 + (64 << 20)
    sv = K.Server(hbm_budget_bytes=one, max_slots=4)
    try:
        t1 = [sv.submit(pr1, nd) for nd in _nodes(K, P1, 3, seed=4, tol=1e-6)]
        t2 = [sv.submit(pr2, nd) for nd in _nodes(K, P2, 3, seed=5, tol=1e-6)]
        res = [sv.poll(t, timeout_ms=120000) for t in t1 + t2]
        st = sv.stats()
    finally:
        sv.close()
    assert all(r.status == "ok" and r.rel_gap <= 1e-6 for r in res)
    assert st["peak_bytes"] <= one
    # a budget below one problem: the request is refused, nothing runs
    sv = K.Server(hbm_budget_bytes=1 << 20, max_slots=4)
    try:
        t = sv.submit(pr1, _nodes(K, P1, 1, seed=6)[0])
        with pytest.raises(K.KscError) as e:
            sv.poll(t, timeout_ms=60000)
        assert e.value.status == K.KSC_ERR_ADMISSION
    finally:
        sv.close()


def test_poll_timeout_unknown_ticket_and_latency(K, problems):
    (P1, pr1), _ = problems
    sv = K.Server(hbm_budget_bytes=8 << 30, max_slots=4)
    try:
        nd = _nodes(K, P1, 1, seed=7, tol=1e-9)[0]
        t0 = time.perf_counter()
        t = sv.submit(pr1, nd)
        early = sv.poll(t, timeout_ms=0)
        r = early or sv.poll(t, timeout_ms=120000)
        wall = time.perf_counter() - t0
        assert r.status == "ok"
        lat = sv.latency(t)
        assert 0.0 < lat <= wall + 1e-3
        with pytest.raises(K.KscError):
            sv.poll(t, timeout_ms=0)          # released
        with pytest.raises(K.KscError):
            sv.poll(987654321, timeout_ms=0)  # never issued
    finally:
        sv.close()


def test_fp32_problem_is_served_by_the_single_node_path(K):
    P = G.make_problem(300, 90, r=0.5, seed=33, loss=G.LSQ, k_true=4, x_dtype=G.F32,
                       lambda2=0.5, M=2.0, k=4)
    pr = K.Problem(P.X, P.y)
    nds = _nodes(K, P, 3, seed=8, tol=1e-8)
    sv = K.Server(hbm_budget_bytes=1 << 30, max_slots=4)
    try:
        res = [sv.poll(sv.submit(pr, nd), timeout_ms=120000) for nd in nds]
    finally:
        sv.close()
    for nd, r in zip(nds, res):
        s = pr.solve(nd)
        assert r.dual_bound == s.dual_bound and np.array_equal(r.beta, s.beta)
