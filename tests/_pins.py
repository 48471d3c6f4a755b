"""Independent reference computations that pin the oracle to mathematics.

None of these reuse the oracle's algorithms: they are brute-force solves,
textbook KKT characterisations, enumerations and closed forms derived from the
definitions in the paper (Sec. 2-3).  Tests compare the oracle against them.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy import optimize


def huber_def(a, M):
    """H_M as a Moreau envelope of M|.|: inf_v  M|v| + 1/2 (a - v)^2 (numeric)."""
    r = optimize.minimize_scalar(lambda v: M * abs(v) + 0.5 * (a - v) ** 2,
                                 bounds=(min(0, a) - 1, max(0, a) + 1), method="bounded",
                                 options={"xatol": 1e-13})
    return r.fun


def huber_smooth(a, M):
    """Huber value and derivative for vector input (used inside brute-force solves)."""
    t = np.abs(a)
    val = np.where(t <= M, 0.5 * t * t, M * t - 0.5 * M * M)
    der = np.clip(a, -M, M)
    return val, der


def prox_scalar_numeric(x, c, M):
    """argmin_v 1/2 (v - x)^2 + c H_M(v) by bounded golden-section search."""
    f = lambda v: 0.5 * (v - x) ** 2 + c * huber_smooth(np.array([v]), M)[0][0]
    lo, hi = min(0.0, x) - 1.0, max(0.0, x) + 1.0
    return optimize.minimize_scalar(f, bounds=(lo, hi), method="bounded",
                                    options={"xatol": 1e-14}).x


def gstar_bruteforce(a, k, M):
    """max over |S| <= k of sum_S H_M(a_j) (definition after Lemma 3.1's proof)."""
    h, _ = huber_smooth(np.asarray(a, float), M)
    best = 0.0
    p = len(h)
    for s in range(0, min(k, p) + 1):
        for S in itertools.combinations(range(p), s):
            best = max(best, float(sum(h[list(S)])))
    return best


def g_kkt(beta, k, M):
    """g(beta) = min 1/2 sum b_j^2/z_j over z in [|b|/M, 1], sum z <= k, by the
    continuous-knapsack KKT conditions: z_j = min(1, |b_j|/tau) with tau chosen by
    bisection so that sum z = k (Eq. g definition, Sec. 3)."""
    b = np.abs(np.asarray(beta, float))
    if b.size == 0:
        return 0.0
    if b.max() > M * (1 + 1e-12) or b.sum() > k * M * (1 + 1e-12):
        return np.inf
    nz = b[b > 0]
    if nz.size <= k:
        return 0.5 * float((nz ** 2).sum())
    # tau lies in (0, max(max|b|, sum|b|/k)]: for tau >= max|b| all z = |b|/tau < 1
    lo, hi = 0.0, float(max(nz.max(), nz.sum() / k))
    for _ in range(200):
        tau = 0.5 * (lo + hi)
        if np.minimum(1.0, nz / tau).sum() > k:
            lo = tau
        else:
            hi = tau
    tau = hi
    z = np.minimum(1.0, nz / tau)
    return 0.5 * float((nz ** 2 / z).sum())


def prox_gstar_bruteforce(mu, k, rho, M):
    """argmin_a 1/2||a - mu||^2 + rho * max_{|S|=k} sum_S H_M(a_j), as a smooth
    epigraph program over (a, t) solved by SLSQP (tiny p only)."""
    mu = np.asarray(mu, float)
    p = mu.size
    subsets = list(itertools.combinations(range(p), min(k, p)))

    def obj(x):
        return 0.5 * np.sum((x[:p] - mu) ** 2) + rho * x[p]

    def obj_jac(x):
        g = np.zeros(p + 1)
        g[:p] = x[:p] - mu
        g[p] = rho
        return g

    cons = []
    for S in subsets:
        S = list(S)

        def c(x, S=S):
            v, _ = huber_smooth(x[S], M)
            return x[p] - v.sum()

        def cj(x, S=S):
            _, d = huber_smooth(x[S], M)
            J = np.zeros(p + 1)
            J[S] = -d
            J[p] = 1.0
            return J

        cons.append({"type": "ineq", "fun": c, "jac": cj})
    h0, _ = huber_smooth(mu, M)
    x0 = np.concatenate([mu * 0.5, [np.sort(h0)[::-1][:k].sum()]])
    r = optimize.minimize(obj, x0, jac=obj_jac, constraints=cons, method="SLSQP",
                          options={"ftol": 1e-15, "maxiter": 2000})
    return r.x[:p]


def naive_pava(m, wts, M):
    """Generic PAVA for min sum_j 1/2(v_j - m_j)^2 + wts_j H_M(v_j) s.t. v
    non-increasing: merge any adjacent violating pair, block values by a 1-D
    numeric minimisation (no closed form, no look-ahead)."""
    blocks = [[j] for j in range(len(m))]

    def value(B):
        f = lambda v: sum(0.5 * (v - m[j]) ** 2 + wts[j] * huber_smooth(np.array([v]), M)[0][0]
                          for j in B)
        lo = min(0.0, min(m[j] for j in B)) - 1
        hi = max(m[j] for j in B) + 1
        return optimize.minimize_scalar(f, bounds=(lo, hi), method="bounded",
                                        options={"xatol": 1e-14}).x

    vals = [value(B) for B in blocks]
    changed = True
    while changed:
        changed = False
        for i in range(len(blocks) - 1):
            if vals[i] < vals[i + 1] - 1e-13:
                blocks[i] = blocks[i] + blocks[i + 1]
                del blocks[i + 1]
                vals[i] = value(blocks[i])
                del vals[i + 1]
                changed = True
                break
    out = np.zeros(len(m))
    for B, v in zip(blocks, vals):
        out[B] = v
    return out


def prox_threshold_form(w, k, rho, M):
    """prox_{rho^-1 g}(w) by the single-pooled-block threshold characterisation
    (the reading used by the GPU kernel): top-k |w| get
    min(M, rho|w|/(1+rho), |w| - theta), the rest max(0, |w| - theta), with theta
    the root of the monotone piecewise-linear
      Phi(t) = sum_top (t + min(rho t, M) - a)_+ - sum_tail (a - t)_+ ."""
    w = np.asarray(w, float)
    a = np.abs(w)
    p = a.size
    order = np.lexsort((np.arange(p), -a))
    k = min(k, p)
    top, tail = order[:k], order[k:]

    def Phi(t):
        s = np.sum(np.maximum(0.0, t + np.minimum(rho * t, M) - a[top]))
        return s - np.sum(np.maximum(0.0, a[tail] - t))

    bps = [0.0, M / rho]
    for x in a[top]:
        bps.append(x / (1 + rho) if x <= M * (1 + rho) / rho else x - M)
    bps.extend(a[tail])
    bps.append(a.max() if p else 0.0)
    bps = np.unique(np.asarray(bps))
    vals = np.array([Phi(t) for t in bps])
    if np.any(vals == 0):
        theta = bps[np.nonzero(vals == 0)[0][0]]
    else:
        i = np.nonzero(vals < 0)[0].max()
        lo, hi = bps[i], bps[i + 1]
        theta = lo - vals[i] * (hi - lo) / (vals[i + 1] - vals[i])
    mag = np.maximum(0.0, a - theta)
    mag[top] = np.minimum(np.minimum(M, rho * a[top] / (1 + rho)), a[top] - theta)
    return np.sign(w) * mag, theta


def ridge_box(X, y, lam, M, loss=0):
    """min F(X b) + lam ||b||^2 s.t. |b| <= M (least squares via bounded LS,
    logistic and squared hinge via L-BFGS-B)."""
    n, s = X.shape
    if s == 0:
        return float({0: y @ y, 1: n * np.log(2.0), 2: n, 3: n, 4: y.sum()}[loss]), np.zeros(0)
    if loss == 0:
        A = np.vstack([X, np.sqrt(lam) * np.eye(s)])
        rhs = np.concatenate([y, np.zeros(s)])
        r = optimize.lsq_linear(A, rhs, bounds=(-M, M), method="bvls", tol=1e-15)
        b = r.x
        return float(np.sum((X @ b - y) ** 2) + lam * b @ b), b

    def f(b):
        if loss == 2:                      # squared hinge, C^1: L-BFGS-B still applies
            m = np.maximum(0.0, 1.0 - y * (X @ b))
            return float(m @ m + lam * b @ b), X.T @ (-2.0 * y * m) + 2 * lam * b
        if loss == 3:                      # Poisson: e^u - y u
            u = X @ b
            e = np.exp(u)
            return float(np.sum(e - y * u) + lam * b @ b), X.T @ (e - y) + 2 * lam * b
        if loss == 4:                      # Gamma: y e^-u + u
            u = X @ b
            e = y * np.exp(-u)
            return float(np.sum(e + u) + lam * b @ b), X.T @ (1.0 - e) + 2 * lam * b
        t = -y * (X @ b)
        v = np.logaddexp(0, t).sum() + lam * b @ b
        sg = 1.0 / (1.0 + np.exp(-t))
        g = X.T @ (-y * sg) + 2 * lam * b
        return v, g

    r = optimize.minimize(f, np.zeros(s), jac=True, method="L-BFGS-B",
                          bounds=[(-M, M)] * s, options={"ftol": 1e-16, "gtol": 1e-12,
                                                         "maxiter": 10000})
    return float(r.fun), r.x


def mip_enumerate(X, y, lam, M, k, loss=0, zero=(), one=()):
    """P_MIP* of the node (all supports of size <= k that contain `one` and avoid
    `zero`), each support solved as a box-constrained ridge problem."""
    p = X.shape[1]
    zero, one = set(zero), set(one)
    free = [j for j in range(p) if j not in zero and j not in one]
    best = np.inf
    kp = k - len(one)
    for s in range(0, max(kp, 0) + 1):
        for S in itertools.combinations(free, s):
            cols = sorted(list(one) + list(S))
            v, _ = ridge_box(X[:, cols], y, lam, M, loss)
            best = min(best, v)
    return best


def l1_relaxation(X, y, lam, M, k, iters=20000):
    """min ||Xb - y||^2 + lam ||b||^2 s.t. ||b||_1 <= kM, ||b||_inf <= M (App. C),
    by accelerated projected gradient with the exact projection onto the set."""
    n, p = X.shape
    L = 2 * (np.linalg.norm(X, 2) ** 2 + lam)

    def proj(v):
        a = np.abs(v)
        c = np.minimum(a, M)
        if c.sum() <= k * M:
            return np.sign(v) * c
        lo, hi = 0.0, a.max()
        for _ in range(200):
            t = 0.5 * (lo + hi)
            if np.clip(a - t, 0, M).sum() > k * M:
                lo = t
            else:
                hi = t
        return np.sign(v) * np.clip(a - hi, 0, M)

    b = np.zeros(p)
    bp = b.copy()
    for t in range(1, iters + 1):
        z = b + (t - 1) / (t + 2) * (b - bp)
        g = 2 * X.T @ (X @ z - y) + 2 * lam * z
        bp = b
        b = proj(z - g / L)
    return float(np.sum((X @ b - y) ** 2) + lam * b @ b)


def conj_numeric(loss, zeta, y):
    """-F*(-zeta) = inf_u F(u) + zeta^T u, coordinate-wise, by 1-D minimisation."""
    tot = 0.0
    for zi, yi in zip(zeta, y):
        if loss == 0:
            f = lambda u: (u - yi) ** 2 + zi * u
        elif loss == 2:
            f = lambda u: max(0.0, 1.0 - yi * u) ** 2 + zi * u
        elif loss == 3:
            f = lambda u: np.exp(u) - yi * u + zi * u
        elif loss == 4:
            f = lambda u: yi * np.exp(-u) + u + zi * u
        else:
            f = lambda u: np.logaddexp(0, -yi * u) + zi * u
        r = optimize.minimize_scalar(f, bounds=(-60, 60), method="bounded",
                                     options={"xatol": 1e-13})
        tot += r.fun
    return tot
