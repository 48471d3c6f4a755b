"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test compares the oracle with a computation that does not share its
algorithm (brute force, KKT characterisation, enumeration, closed form), so a
dropped term, wrong sign, wrong index or transposed operand in the oracle fails
at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import _pins as P

RNG = np.random.default_rng(12345)


# ------------------------------------------------------------------ Huber (Sec. 3.1)

@pytest.mark.parametrize("a", [-7.5, -2.0, -0.3, 0.0, 0.7, 1.99, 2.0, 2.01, 9.0])
@pytest.mark.parametrize("M", [0.5, 2.0])
def test_huber_is_moreau_envelope_of_abs(a, M):
    # H_M(a) = inf_v M|v| + (a-v)^2/2: an independent characterisation
    assert abs(O.huber(a, M) - P.huber_def(a, M)) < 1e-10


@pytest.mark.parametrize("x", [-9.0, -3.0, -0.4, 0.0, 0.4, 2.9, 3.0, 3.1, 12.0])
@pytest.mark.parametrize("c", [0.0, 0.5, 2.0])
def test_huber_prox_vs_golden_section(x, c):
    M = 1.0
    # golden-section search resolves the minimiser to ~sqrt(eps) at the kink x = M(1+c)
    assert abs(O.huber_prox(x, c, M) - P.prox_scalar_numeric(x, c, M)) < 1e-7


# --------------------------------------------------- prox of g* (Alg 1 + Alg 4)

@pytest.mark.parametrize("case", range(12))
def test_prox_gstar_vs_bruteforce_convex_solve(case):
    rng = np.random.default_rng(100 + case)
    p = int(rng.integers(2, 7))
    k = int(rng.integers(1, p + 1))
    rho = float(rng.choice([0.3, 1.0, 3.0]))
    M = float(rng.choice([0.5, 1.0, 4.0]))
    mu = rng.standard_normal(p) * 3
    al, _ = O.prox_gstar(mu, k, rho, M)
    ref = P.prox_gstar_bruteforce(mu, k, rho, M)
    assert np.max(np.abs(al - ref)) < 2e-5, (al, ref)


def _check_fenchel_young(w, k, rho, M, beta):
    alpha = rho * (w - beta)
    g = P.g_kkt(beta, k, M)
    gs = P.gstar_bruteforce(alpha, k, M) if w.size <= 10 else _gstar_sorted(alpha, k, M)
    lhs = g + gs
    rhs = float(beta @ alpha)
    return abs(lhs - rhs) / max(1.0, abs(rhs))


def _gstar_sorted(a, k, M):
    h, _ = P.huber_smooth(a, M)
    return float(np.sort(h)[::-1][:k].sum())


@pytest.mark.parametrize("case", range(40))
def test_prox_g_fenchel_young_certificate(case):
    # beta = prox_{rho^-1 g}(w)  <=>  alpha = rho (w - beta) in dg(beta)
    # <=> g(beta) + g*(alpha) = beta^T alpha   (exact optimality certificate)
    rng = np.random.default_rng(200 + case)
    p = int(rng.integers(1, 60))
    k = int(rng.integers(1, p + 2))   # k = 0 is pinned by test_prox_k_zero_is_zero
    rho = float(10 ** rng.uniform(-1.5, 2.5))
    M = float(10 ** rng.uniform(-1, 1))
    w = rng.standard_normal(p) * (10 ** rng.uniform(-1, 1))
    beta, _ = O.prox_g(w, k, rho, M)
    assert _check_fenchel_young(w, k, rho, M, beta) < 1e-11


def test_prox_preserves_sign_and_order():
    for case in range(30):
        rng = np.random.default_rng(300 + case)
        p = int(rng.integers(2, 200))
        mu = rng.standard_normal(p) * 4
        al, _ = O.prox_gstar(mu, int(rng.integers(0, p)), 1.7, 1.3)
        assert np.all(al * mu >= 0)
        o = np.argsort(-np.abs(mu), kind="stable")
        assert np.all(np.diff(np.abs(al[o])) <= 1e-15)


def test_prox_k_equals_p_is_ridge_clip():
    # k >= p: g = 1/2||b||^2 on the box, so prox_{rho^-1 g}(w) = clip(rho w/(1+rho), +-M)
    for case in range(10):
        rng = np.random.default_rng(400 + case)
        p = int(rng.integers(1, 50))
        w = rng.standard_normal(p) * 3
        rho, M = 2.5, 1.1
        beta, _ = O.prox_g(w, p, rho, M)
        assert np.allclose(beta, np.clip(rho * w / (1 + rho), -M, M), rtol=0, atol=1e-14)


def test_prox_k_zero_is_zero():
    w = RNG.standard_normal(17)
    beta, _ = O.prox_g(w, 0, 3.0, 1.0)
    assert np.all(np.abs(beta) < 1e-14)


@pytest.mark.parametrize("case", range(10))
def test_alg4_merge_equals_naive_pava(case):
    rng = np.random.default_rng(500 + case)
    p = int(rng.integers(2, 14))
    k = int(rng.integers(1, p + 1))
    rho, M = float(rng.uniform(0.2, 5)), float(rng.uniform(0.3, 3))
    mu = rng.standard_normal(p) * 3
    al, perm = O.prox_gstar(mu, k, rho, M)
    m = np.abs(mu)[perm]
    wts = np.array([rho if r < k else 0.0 for r in range(p)])
    nu = P.naive_pava(m, wts, M)
    # block values from a bounded 1-D minimiser: resolved to ~sqrt(eps) relative
    assert np.max(np.abs(np.abs(al)[perm] - nu)) < 3e-7 * max(1.0, np.abs(mu).max())


def test_moreau_identity_and_threshold_form():
    # the GPU kernel's reading (one pooled block, threshold theta) equals Alg 1+4
    for case in range(300):
        rng = np.random.default_rng(600 + case)
        p = int(rng.integers(1, 80))
        k = int(rng.integers(0, p + 1))
        rho = float(10 ** rng.uniform(-2, 3))
        M = float(10 ** rng.uniform(-1, 1))
        w = rng.standard_normal(p) * (10 ** rng.uniform(-2, 1))
        if case % 7 == 0:  # ties
            w = np.round(w, 1)
        beta, _ = O.prox_g(w, k, rho, M)
        thr, _ = P.prox_threshold_form(w, k, rho, M)
        scale = max(1.0, np.abs(w).max())
        assert np.max(np.abs(beta - thr)) <= 1e-12 * scale * max(1.0, rho)
        # Moreau: w = prox_{rho^-1 g}(w) + rho^-1 prox_{rho g*}(rho w)
        al, _ = O.prox_gstar(rho * w, k, rho, M)
        assert np.max(np.abs(w - beta - al / rho)) <= 1e-12 * scale


def test_prox_sort_order_is_stable_descending():
    mu = np.array([1.0, -3.0, 3.0, 0.5, -1.0, 3.0])
    _, perm = O.prox_gstar(mu, 2, 1.0, 1.0)
    assert list(perm) == [1, 2, 5, 0, 4, 3]


# --------------------------------------------------------------- g (Alg 2)

@pytest.mark.parametrize("case", range(60))
def test_g_value_vs_kkt_waterfilling(case):
    rng = np.random.default_rng(700 + case)
    p = int(rng.integers(1, 100))
    k = int(rng.integers(1, p + 3))
    M = float(rng.uniform(0.5, 3))
    b = rng.uniform(-1, 1, p) * M
    if b.__abs__().sum() > k * M:
        b *= 0.99 * k * M / np.abs(b).sum()
    if case % 5 == 0:
        b[rng.random(p) < 0.5] = 0.0
    g = O.g_value(b, k, M)
    ref = P.g_kkt(b, k, M)
    assert abs(g - ref) <= 1e-11 * max(1.0, abs(ref))


def test_g_special_cases():
    rng = np.random.default_rng(800)
    # k-sparse feasible beta: z = 1 on the support, g = ||b||^2/2
    b = np.zeros(30)
    b[[3, 7, 11]] = [1.2, -0.4, 0.9]
    assert abs(O.g_value(b, 3, 2.0) - 0.5 * b @ b) < 1e-15
    assert abs(O.g_value(b, 5, 2.0) - 0.5 * b @ b) < 1e-15
    # spread-out beta with max|b| <= ||b||_1/k: g = ||b||_1^2 / (2k)
    b = rng.uniform(0.9, 1.0, 20) * np.where(rng.random(20) < 0.5, -1, 1)
    k = 4
    assert np.abs(b).max() <= np.abs(b).sum() / k
    assert abs(O.g_value(b, k, 10.0) - np.abs(b).sum() ** 2 / (2 * k)) < 1e-12
    # outside dom g
    assert O.g_value(np.array([2.5, 0.0]), 1, 2.0) == math.inf
    assert O.g_value(np.array([1.5, 1.5, 1.5]), 2, 2.0) == math.inf
    assert O.g_value(np.zeros(5), 0, 1.0) == 0.0


def test_relaxed_z_properties():
    for case in range(40):
        rng = np.random.default_rng(900 + case)
        p = int(rng.integers(1, 80))
        k = int(rng.integers(1, p + 1))
        M = 1.5
        b = rng.uniform(-1, 1, p) * M * rng.uniform(0.05, 1)
        if np.abs(b).sum() > k * M:
            b *= 0.9 * k * M / np.abs(b).sum()
        g, z = O.g_value(b, k, M, want_z=True)
        assert np.all(z >= -1e-15) and np.all(z <= 1 + 1e-12)
        assert np.all(np.abs(b) <= M * z + 1e-12)
        if np.abs(b).sum() > 0 and np.count_nonzero(b) > k:
            assert abs(z.sum() - k) < 1e-9
        nz = z > 0
        assert abs(0.5 * np.sum(b[nz] ** 2 / z[nz]) - g) <= 1e-10 * max(1, g)


# --------------------------------------------------------- g* (Lemma 3.1)

@pytest.mark.parametrize("case", range(20))
def test_gstar_vs_subset_bruteforce(case):
    rng = np.random.default_rng(1000 + case)
    p = int(rng.integers(1, 9))
    k = int(rng.integers(0, p + 1))
    M = float(rng.uniform(0.3, 3))
    a = rng.standard_normal(p) * 3
    assert abs(O.gstar(a, k, M) - P.gstar_bruteforce(a, k, M)) < 1e-12


def test_gstar_is_attained_at_lemma_maximiser():
    # beta* = sgn(a) min(|a|, M) z with z the indicator of the top-k H_M (App. A)
    for case in range(20):
        rng = np.random.default_rng(1100 + case)
        p, k, M = 25, int(rng.integers(1, 10)), 1.3
        a = rng.standard_normal(p) * 2
        h, _ = P.huber_smooth(a, M)
        top = np.argsort(-h, kind="stable")[:k]
        bstar = np.zeros(p)
        bstar[top] = np.sign(a[top]) * np.minimum(np.abs(a[top]), M)
        val = a @ bstar - P.g_kkt(bstar, k, M)
        assert abs(val - O.gstar(a, k, M)) < 1e-11
        # Fenchel-Young inequality at random feasible points
        for _ in range(5):
            b = rng.uniform(-M, M, p) * 0.3
            if np.abs(b).sum() > k * M:
                b *= 0.9 * k * M / np.abs(b).sum()
            assert a @ b - P.g_kkt(b, k, M) <= O.gstar(a, k, M) + 1e-11


# ------------------------------------------------------ losses (App. D.1)

@pytest.mark.parametrize("loss", [0, 1, 2])
def test_negative_conjugate_vs_numeric_inf(loss):
    rng = np.random.default_rng(1200 + loss)
    n = 12
    if loss == 0:
        y = rng.standard_normal(n)
        zeta = rng.standard_normal(n)
    elif loss == 1:
        y = np.where(rng.random(n) < 0.5, -1.0, 1.0)
        zeta = y * rng.uniform(0.02, 0.98, n)
    else:
        y = np.where(rng.random(n) < 0.5, -1.0, 1.0)
        zeta = y * rng.uniform(0.0, 3.0, n)
    assert abs(O.neg_conj(loss, zeta, y) - P.conj_numeric(loss, zeta, y)) < 1e-7


def test_squared_hinge_conjugate_domain_and_fenchel_young():
    # outside y zeta >= 0 the infimum of F(u) + zeta^T u is unbounded below; at
    # zeta = -grad F(u) Fenchel-Young holds with equality, elsewhere as >=
    rng = np.random.default_rng(1250)
    n = 15
    y = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    bad = y * rng.uniform(0.0, 2.0, n)
    bad[3] = -0.1 * y[3]
    assert O.neg_conj(2, bad, y) == -np.inf
    u = 2.0 * rng.standard_normal(n)
    zeta = -O.loss_grad(2, u, y)
    assert np.all(y * zeta >= 0)
    assert abs(O.loss(2, u, y) + zeta @ u - O.neg_conj(2, zeta, y)) < 1e-12 * n
    for _ in range(20):
        v = rng.standard_normal(n)
        assert O.loss(2, v, y) + zeta @ v >= O.neg_conj(2, zeta, y) - 1e-12


def test_loss_gradients_by_finite_differences():
    rng = np.random.default_rng(1300)
    n = 9
    for loss in (0, 1, 2):
        y = rng.standard_normal(n) if loss == 0 else np.where(rng.random(n) < .5, -1., 1.)
        u = rng.standard_normal(n)
        if loss == 2:                 # keep off the kink 1 - y u = 0
            u = np.where(np.abs(1 - y * u) < 1e-3, u + 0.01, u)
        g = O.loss_grad(loss, u, y)
        h = 1e-6
        for i in range(n):
            e = np.zeros(n)
            e[i] = h
            fd = (O.loss(loss, u + e, y) - O.loss(loss, u - e, y)) / (2 * h)
            assert abs(fd - g[i]) < 1e-6


def test_matvecs_and_power_iteration():
    rng = np.random.default_rng(1400)
    X = rng.standard_normal((37, 23))
    v = rng.standard_normal(23)
    r = rng.standard_normal(37)
    assert np.allclose(O.matvec(X, v), X @ v, atol=1e-12)
    assert np.allclose(O.rmatvec(X, r), X.T @ r, atol=1e-12)
    assert np.allclose(O.matvec(X.astype(np.float32), v), X.astype(np.float32).astype(float) @ v,
                       atol=1e-12)
    lam, _ = O.power_iteration(X, tol=1e-14)
    assert abs(lam - np.linalg.norm(X, 2) ** 2) < 1e-8 * lam


# ------------------------------------------------------- solver (Alg 3)

def _lsq_problem(n, p, seed, noise=0.3):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    bt = np.zeros(p)
    bt[rng.choice(p, 3, replace=False)] = rng.choice([-1.0, 1.0], 3)
    return X, X @ bt + noise * rng.standard_normal(n)


def test_k_equals_p_reduces_to_ridge_closed_form():
    X, y = _lsq_problem(40, 8, 1)
    lam = 0.7
    r = O.solve(X, y, 0, lam, 1e6, 8, tol=1e-13)
    ref = np.linalg.solve(X.T @ X + lam * np.eye(8), X.T @ y)
    assert r.status == "converged"
    assert np.max(np.abs(r.beta - ref)) < 1e-6
    assert abs(r.primal - (np.sum((X @ ref - y) ** 2) + lam * ref @ ref)) < 1e-9 * r.primal


def test_k_equals_p_with_active_box_matches_bounded_ls():
    X, y = _lsq_problem(40, 8, 2, noise=0.1)
    y = 3 * y
    lam, M = 0.2, 0.8
    r = O.solve(X, y, 0, lam, M, 8, tol=1e-13, max_iter=200000)
    v, b = P.ridge_box(X, y, lam, M)
    assert np.max(np.abs(r.beta - b)) < 1e-6
    assert abs(r.primal - v) < 1e-9 * v


def test_squared_hinge_k_equals_p_is_box_l2_svm():
    # k = p: the perspective term is lambda2 ||b||^2 on the box, so the relaxation
    # is the box-constrained squared-hinge ridge problem (an L2-SVM)
    rng = np.random.default_rng(1450)
    n, p = 40, 7
    X = rng.standard_normal((n, p))
    y = np.where(X[:, 0] - 0.5 * X[:, 1] + 0.4 * rng.standard_normal(n) > 0, 1.0, -1.0)
    lam, M = 0.3, 0.6
    r = O.solve(X, y, 2, lam, M, p, tol=1e-13, max_iter=200000)
    v, b = P.ridge_box(X, y, lam, M, loss=2)
    assert r.status == "converged"
    assert abs(r.primal - v) < 1e-8 * v
    assert np.max(np.abs(r.beta - b)) < 1e-4


@pytest.mark.parametrize("loss", [0, 1, 2])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_weak_duality_against_mip_enumeration(loss, seed):
    rng = np.random.default_rng(1500 + seed)
    n, p, k = 30, 9, 3
    X = rng.standard_normal((n, p))
    bt = np.zeros(p)
    bt[rng.choice(p, 3, replace=False)] = 1.0
    if loss == 0:
        y = X @ bt + 0.5 * rng.standard_normal(n)
    else:
        y = np.where(rng.random(n) < 1 / (1 + np.exp(-X @ bt)), 1.0, -1.0)
    lam, M = 0.5, 1.5
    r = O.solve(X, y, loss, lam, M, k, tol=1e-12, max_iter=100000)
    mip = P.mip_enumerate(X, y, lam, M, k, loss)
    assert r.status == "converged"
    assert r.dual <= r.primal + 1e-12 * abs(r.primal)
    assert r.dual <= mip + 1e-9 * abs(mip)
    assert r.primal <= mip + 1e-9 * abs(mip)   # relaxation below the MIP optimum


@pytest.mark.parametrize("seed", [0, 1])
def test_node_bound_against_node_enumeration(seed):
    rng = np.random.default_rng(1600 + seed)
    n, p, k = 25, 10, 4
    X = rng.standard_normal((n, p))
    y = X[:, :3].sum(1) + 0.3 * rng.standard_normal(n)
    state = np.zeros(p, np.int8)
    zero, one = [1, 6], [2]
    state[zero] = O.ZERO
    state[one] = O.ONE
    lam, M = 0.3, 2.0
    r = O.solve(X, y, 0, lam, M, k, state=state, tol=1e-12, max_iter=100000)
    mip = P.mip_enumerate(X, y, lam, M, k, 0, zero=zero, one=one)
    assert r.status == "converged"
    assert np.all(r.beta[zero] == 0)
    assert r.dual <= mip + 1e-9 * mip and r.primal <= mip + 1e-9 * mip
    # the node problem with no free budget and S1 = true support is a ridge on S1
    st = np.full(p, O.ZERO, np.int8)
    st[[0, 1, 2]] = O.ONE
    r2 = O.solve(X, y, 0, lam, M, 3, state=st, tol=1e-13, max_iter=100000)
    v, b = P.ridge_box(X[:, [0, 1, 2]], y, lam, M)
    assert abs(r2.primal - v) < 1e-9 * v
    assert np.max(np.abs(r2.beta[[0, 1, 2]] - b)) < 1e-6


def test_perspective_bound_not_below_l1_relaxation():
    # App. C: the perspective relaxation is at least as tight as the l1 one
    X, y = _lsq_problem(30, 12, 3, noise=0.5)
    lam, M, k = 0.5, 1.2, 3
    r = O.solve(X, y, 0, lam, M, k, tol=1e-12, max_iter=100000)
    l1 = P.l1_relaxation(X, y, lam, M, k)
    assert r.primal >= l1 - 1e-7 * l1


def test_restart_beats_plain_fista_and_ista():
    # Fig. 3 (qualitative): restarted FISTA reaches a tight gap in far fewer iterations
    X, y = _lsq_problem(80, 40, 4, noise=0.5)
    kw = dict(tol=1e-9, max_iter=50000)
    a = O.solve(X, y, 0, 0.5, 2.0, 4, **kw)
    b = O.solve(X, y, 0, 0.5, 2.0, 4, restart=False, **kw)
    c = O.solve(X, y, 0, 0.5, 2.0, 4, restart=False, momentum=False, **kw)
    assert a.status == "converged"
    assert a.iters < b.iters and a.iters < c.iters
    assert abs(a.primal - b.primal) < 1e-7 * a.primal


def test_incumbent_rules():
    X, y = _lsq_problem(50, 12, 5)
    r = O.solve(X, y, 0, 0.5, 2.0, 3, tol=1e-12)
    pr = O.solve(X, y, 0, 0.5, 2.0, 3, incumbent=r.dual * 0.5)
    assert pr.status == "pruned" and pr.dual > r.dual * 0.5
    lo = O.solve(X, y, 0, 0.5, 2.0, 3, incumbent=r.primal * 1.5)
    assert lo.status == "primal_below" and lo.primal < r.primal * 1.5
    st = np.zeros(12, np.int8)
    st[:4] = O.ONE
    inf = O.solve(X, y, 0, 0.5, 2.0, 3, state=st)
    assert inf.status == "infeasible" and inf.dual == math.inf


def test_dual_bound_is_valid_at_any_iterate():
    X, y = _lsq_problem(40, 15, 6)
    r = O.solve(X, y, 0, 0.4, 1.5, 3, tol=1e-12, max_iter=3000, want_trace=True)
    assert np.all(r.trace[:, 1] <= r.primal + 1e-10 * r.primal)
    # any beta gives a valid bound
    rng = np.random.default_rng(7)
    for _ in range(5):
        b = rng.standard_normal(15) * 0.3
        assert O.dual_bound(X, y, 0, 0.4, 1.5, 3, b) <= r.primal + 1e-10 * r.primal


# ------------------------------------------- eigen-perspective bound (App. D.2)

def _eig_problem(seed, n=40, p=8, k=3, noise=0.4):
    rng = np.random.default_rng(1700 + seed)
    X = rng.standard_normal((n, p))
    X[:, 1] += 0.6 * X[:, 0]            # correlated columns: lambda_min well below the mean
    bt = np.zeros(p)
    bt[rng.choice(p, k, replace=False)] = rng.choice([-1.0, 1.0], k)
    return X, X @ bt + noise * rng.standard_normal(n), rng


def test_lambda_min_is_the_smallest_eigenvalue():
    X, _, rng = _eig_problem(0)
    lam = O.lambda_min(X)
    A = X.T @ X
    # positive semidefinite at lambda_min and not above it (Rayleigh quotients)
    assert np.all(np.linalg.eigvalsh(A - lam * np.eye(8)) >= -1e-9 * lam)
    for _ in range(50):
        v = rng.standard_normal(8)
        assert v @ A @ v / (v @ v) >= lam * (1 - 1e-12)
    assert O.lambda_min(rng.standard_normal((5, 9))) == 0.0   # n < p: singular


def test_eig_bound_at_lambda_to_zero_is_the_perspective_bound():
    # the eigen bound's lambda-free part is the Sec. 3.4 bound for least squares
    X, y, rng = _eig_problem(1)
    for _ in range(5):
        b = rng.uniform(-1, 1, 8)
        for st in (None, np.array([0, 1, 0, 2, 0, 0, 1, 0], np.int8)):
            d0 = O.dual_bound(X, y, 0, 0.6, 1.5, 3, b, state=st)
            de = O.dual_bound(X, y, 0, 0.6, 1.5, 3, b, state=st, eig=1e-9)
            assert abs(de - d0) <= 1e-7 * (1 + abs(d0))


def test_eig_relaxation_at_k_equals_p_is_the_box_ridge_problem():
    # with k = p, 2 lambda_eig g(b) = lambda_eig ||b||^2 on the box, so the eigen
    # relaxation's objective is ||X b - y||^2 + lambda2 ||b||^2 itself
    X, y, _ = _eig_problem(2)
    y = 2.5 * y
    lam, M = 0.3, 0.7
    eig = 0.9 * O.lambda_min(X)
    r = O.solve(X, y, 0, lam, M, 8, tol=1e-13, max_iter=200000, eig=eig)
    v, b = P.ridge_box(X, y, lam, M)
    assert r.status == "converged"
    assert abs(r.primal - v) < 1e-9 * v and abs(r.dual - v) < 1e-9 * v
    assert np.max(np.abs(r.beta - b)) < 1e-6


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_eig_bound_is_valid_and_tighter_than_the_perspective_bound(seed):
    X, y, rng = _eig_problem(seed)
    lam, M, k = 0.4, 1.5, 3
    eig = O.lambda_min(X)
    mip = P.mip_enumerate(X, y, lam, M, k, 0)
    persp = O.solve(X, y, 0, lam, M, k, tol=1e-12, max_iter=200000)
    r = O.solve(X, y, 0, lam, M, k, tol=1e-12, max_iter=200000, eig=eig)
    assert r.status == "converged"
    assert r.dual <= mip + 1e-9 * abs(mip)          # weak duality against P_MIP*
    assert r.primal <= mip + 1e-9 * abs(mip)        # still a relaxation
    assert r.dual >= persp.dual + 1e-3 * abs(mip)   # P_eig* > P_persp* on these instances
    # a smaller shift interpolates between the two relaxations
    r2 = O.solve(X, y, 0, lam, M, k, tol=1e-12, max_iter=200000, eig=0.5 * eig)
    assert persp.dual - 1e-9 * abs(mip) <= r2.dual <= r.dual + 1e-9 * abs(mip)
    # the bound holds at any point, not only at the optimum
    for _ in range(10):
        b = rng.uniform(-M, M, 8)
        assert O.dual_bound(X, y, 0, lam, M, k, b, eig=eig) <= mip + 1e-9 * abs(mip)


def test_eig_node_bound_against_node_enumeration():
    X, y, _ = _eig_problem(6, p=9)
    lam, M, k = 0.3, 2.0, 3
    st = np.zeros(9, np.int8)
    st[[2, 5]] = O.ZERO
    st[[0]] = O.ONE
    eig = O.lambda_min(X)
    mip = P.mip_enumerate(X, y, lam, M, k, 0, zero=(2, 5), one=(0,))
    r = O.solve(X, y, 0, lam, M, k, state=st, tol=1e-12, max_iter=200000, eig=eig)
    rp = O.solve(X, y, 0, lam, M, k, state=st, tol=1e-12, max_iter=200000)
    assert r.status == "converged"
    assert rp.dual - 1e-9 * abs(mip) <= r.dual <= mip + 1e-9 * abs(mip)
    assert r.beta[2] == 0 and r.beta[5] == 0


def test_eig_bound_is_the_mip_optimum_for_orthogonal_columns():
    # X^T X = n I: with lambda = n the eigen relaxation is separable and tight --
    # 2 lambda_eig H_M(|c_j| / lambda_eig), c = X^T y, is the best decrease
    # 2 |c_j| b_j - (n + lambda2) b_j^2 of one coordinate, so the bound equals the
    # closed-form optimum of Eq. (1): ||y||^2 minus the k largest decreases
    rng = np.random.default_rng(1800)
    n, p, k = 30, 8, 3
    Qm, _ = np.linalg.qr(rng.standard_normal((n, p)))
    X = np.sqrt(n) * Qm
    bt = np.zeros(p)
    bt[[1, 4, 6]] = [1.0, -1.0, 0.5]
    y = X @ bt + 0.3 * rng.standard_normal(n)
    lam, M = 0.5, 0.9
    c = X.T @ y
    b = np.minimum(np.abs(c) / (n + lam), M)
    dec = 2 * np.abs(c) * b - (n + lam) * b * b
    closed = float(y @ y - np.sort(dec)[-k:].sum())
    assert abs(closed - P.mip_enumerate(X, y, lam, M, k, 0)) <= 1e-9 * closed
    # Q = X^T X - lambda I is (numerically) 0, so the bound does not depend on b
    eig = n * (1 - 1e-12)
    for beta in (np.zeros(p), rng.uniform(-M, M, p), bt):
        assert abs(O.dual_bound(X, y, 0, lam, M, k, beta, eig=eig) - closed) <= 1e-8 * closed
    persp = O.solve(X, y, 0, lam, M, k, tol=1e-12, max_iter=100000)
    assert persp.dual < closed - 1e-3 * closed    # the perspective relaxation is not tight here


# ------------------------------------------- Poisson and Gamma regression (App. D.1)

def _count_problem(loss, n, p, seed, k_true=3):
    """Unit-norm columns, log link (as the input generator draws them)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, p))
    X /= np.linalg.norm(X, axis=0)
    bt = np.zeros(p)
    bt[rng.choice(p, k_true, replace=False)] = rng.choice([-3.0, 3.0], k_true)
    mu = np.exp(X @ bt)
    y = rng.poisson(mu).astype(float) if loss == 3 else rng.gamma(2.0, mu / 2.0)
    return X, y


@pytest.mark.parametrize("loss", [3, 4])
def test_count_losses_conjugate_vs_numeric_inf(loss):
    # -F*(-zeta) = inf_u F(u) + zeta^T u, inside the conjugate's domain
    rng = np.random.default_rng(1600 + loss)
    n = 12
    if loss == 3:
        y = rng.poisson(2.0, n).astype(float)
        zeta = y - rng.uniform(0.05, 4.0, n)          # y - zeta > 0
    else:
        y = rng.gamma(2.0, 1.0, n)
        zeta = rng.uniform(-0.95, 3.0, n)             # 1 + zeta > 0
    assert abs(O.neg_conj(loss, zeta, y) - P.conj_numeric(loss, zeta, y)) < 1e-7


@pytest.mark.parametrize("loss", [3, 4])
def test_count_losses_domain_fenchel_young_and_gradients(loss):
    rng = np.random.default_rng(1650 + loss)
    n = 14
    y = rng.poisson(1.5, n).astype(float) if loss == 3 else rng.gamma(2.0, 1.0, n)
    # outside the domain the infimum is unbounded below
    bad = np.zeros(n)
    if loss == 3:
        bad[:] = y - 1.0
        bad[2] = y[2] + 0.5                            # y - zeta < 0
    else:
        bad[:] = 0.5
        bad[4] = -1.5                                  # 1 + zeta < 0
    assert O.neg_conj(loss, bad, y) == -np.inf
    # at zeta = -grad F(u): Fenchel-Young with equality, elsewhere >=
    u = 0.7 * rng.standard_normal(n)
    zeta = -O.loss_grad(loss, u, y)
    assert abs(O.loss(loss, u, y) + zeta @ u - O.neg_conj(loss, zeta, y)) < 1e-12 * n
    for _ in range(20):
        v = rng.standard_normal(n)
        assert O.loss(loss, v, y) + zeta @ v >= O.neg_conj(loss, zeta, y) - 1e-12
    # gradient by central differences
    g = O.loss_grad(loss, u, y)
    h = 1e-6
    for i in range(n):
        e = np.zeros(n)
        e[i] = h
        fd = (O.loss(loss, u + e, y) - O.loss(loss, u - e, y)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i]))


@pytest.mark.parametrize("loss", [3, 4])
def test_count_losses_k_equals_p_is_box_ridge_glm(loss):
    # k = p: the relaxation is the box-constrained ridge Poisson / Gamma regression
    X, y = _count_problem(loss, 60, 6, 1700 + loss)
    lam, M = 0.3, 1.5
    r = O.solve(X, y, loss, lam, M, 6, tol=1e-13, max_iter=200000)
    v, b = P.ridge_box(X, y, lam, M, loss=loss)
    assert r.status == "converged"
    assert abs(r.primal - v) < 1e-8 * abs(v)
    assert np.max(np.abs(r.beta - b)) < 1e-5


@pytest.mark.parametrize("loss", [3, 4])
@pytest.mark.parametrize("seed", [0, 1])
def test_count_losses_weak_duality_against_mip_enumeration(loss, seed):
    X, y = _count_problem(loss, 40, 8, 1750 + 10 * loss + seed)
    lam, M, k = 0.4, 2.0, 3
    r = O.solve(X, y, loss, lam, M, k, tol=1e-12, max_iter=200000)
    mip = P.mip_enumerate(X, y, lam, M, k, loss)
    assert r.status == "converged"
    assert r.dual <= r.primal + 1e-9 * abs(r.primal)
    assert r.primal <= mip * (1 + 1e-9)
    # with fixed sets
    st = np.zeros(8, np.int8)
    st[[1, 5]] = O.ZERO
    st[2] = O.ONE
    rn = O.solve(X, y, loss, lam, M, k, state=st, tol=1e-12, max_iter=200000)
    mipn = P.mip_enumerate(X, y, lam, M, k, loss, zero=[1, 5], one=[2])
    assert rn.dual <= rn.primal + 1e-9 * abs(rn.primal) and rn.primal <= mipn * (1 + 1e-9)
    assert rn.dual >= r.dual - 1e-9 * abs(r.dual)     # a child's bound is not below the root's optimum


@pytest.mark.parametrize("loss", [3, 4])
def test_count_losses_curvature_bound_holds_where_the_iteration_steps(loss):
    # the step constant of reading R22 bounds the Hessian X^T diag(F'') X at any point
    # within three times the largest |x_i^T b| of the box-and-l1 set
    X, y = _count_problem(loss, 50, 10, 1800 + loss)
    lam, M, k = 0.5, 1.2, 3
    L = O.solve(X, y, loss, lam, M, k, tol=1e-6, max_iter=5).L
    rng = np.random.default_rng(3)
    for _ in range(50):
        b = rng.uniform(-M, M, 10)
        b *= min(1.0, k * M / np.abs(b).sum())
        bp = rng.uniform(-M, M, 10)
        bp *= min(1.0, k * M / np.abs(bp).sum())
        c = rng.uniform(0.0, 1.0)
        g = b + c * (b - bp)                              # an extrapolated point
        u = X @ g
        curv = np.exp(u) if loss == 3 else y * np.exp(-u)
        H = X.T @ (curv[:, None] * X)
        assert np.linalg.eigvalsh(H)[-1] <= L * (1 + 1e-9)
