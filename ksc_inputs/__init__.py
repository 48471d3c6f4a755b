"""Seeded synthetic inputs shaped like the paper's workloads (App. B.2).

This module is shared by the tests, the benchmark and both sides of every
parity check.  It holds none of the solver's arithmetic: it only draws design
matrices (AR(1) Toeplitz rows, standardised columns), sparse +-1 ground truths,
labels, branch-and-bound fixed sets and warm-start perturbations.

Every draw comes from Philox4x32-10 (``gen.c``) keyed by (seed, stream), so a
workload is a pure function of its parameters and seed.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_OUT = os.path.join(_HERE, "_build", "libksc_gen.so")
_lib = None

LSQ, LOGISTIC, SQHINGE = 0, 1, 2   # labels +-1 for the last two
POISSON, GAMMA = 3, 4               # counts >= 0; positive reals
F64, F32, BF16 = "f64", "f32", "bf16"
_DT_CODE = {F64: 0, F32: 1, BF16: 2}

# stream ids (second Philox key word)
_S_SUPPORT, _S_SIGN, _S_NOISE, _S_LABEL, _S_NODES, _S_WARM = 2, 3, 4, 5, 6, 7
_S_MIX, _S_ARRIVAL = 8, 9
_S_COUNT = 10


def build(force: bool = False) -> str:
    stale = not os.path.exists(_OUT) or os.path.getmtime(_SRC) > os.path.getmtime(_OUT)
    if force or stale:
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.ksg_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                           C.POINTER(C.c_uint32)]
        _lib.ksg_uniform.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.POINTER(C.c_double)]
        _lib.ksg_normal.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.POINTER(C.c_double)]
        _lib.ksg_make_X.argtypes = [C.c_int64, C.c_int64, C.c_double, C.c_uint64, C.c_int,
                                    C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.c_int]
    return _lib


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    _L().ksg_philox4x32_10(c, k, o)
    return list(o)


def uniform(seed, stream, count):
    out = np.zeros(count)
    if count:
        _L().ksg_uniform(seed, stream, count, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def normal(seed, stream, count):
    out = np.zeros(count)
    if count:
        _L().ksg_normal(seed, stream, count, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def bf16_to_f32(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32)


def _choose(seed, stream, p, count, salt=0):
    """count distinct indices of [0, p) by a partial Fisher-Yates shuffle."""
    u = uniform(seed + (salt << 20), stream, count)
    perm = np.arange(p)
    for t in range(count):
        j = t + int(u[t] * (p - t))
        perm[t], perm[j] = perm[j], perm[t]
    return perm[:count].copy()


def _threads():
    return max(1, min(32, os.cpu_count() or 1))


@dataclass
class Problem:
    """One synthetic GLM instance.  ``X`` is stored in ``x_dtype`` (bf16 as uint16 bits)."""
    X: np.ndarray
    y: np.ndarray
    beta_star: np.ndarray
    loss: int
    lambda2: float
    M: float
    k: int
    x_dtype: str
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def p(self):
        return self.X.shape[1]

    def X64(self):
        """The stored matrix promoted exactly to float64 (what the oracle solves)."""
        if self.x_dtype == BF16:
            return bf16_to_f32(self.X).astype(np.float64)
        return self.X.astype(np.float64)


def f64_to_bf16(x: np.ndarray) -> np.ndarray:
    """BF16 bits (uint16) of x rounded to nearest, ties to even (via FP32)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def _poisson(mu, u):
    """Poisson(mu) draws by inversion of the CDF at the uniforms u."""
    k = np.zeros(mu.shape)
    pk = np.exp(-mu)
    cdf = pk.copy()
    for j in range(1, 400):
        more = u > cdf
        if not more.any():
            break
        k += more
        pk = pk * mu / j
        cdf = cdf + pk
    return k


def make_problem(n, p, *, r=0.5, seed=0, loss=LSQ, k_true=5, snr=5.0, x_dtype=F64,
                 lambda2=1.0, M=2.0, k=5) -> Problem:
    """Rows ~ N(0, Toeplitz r^|j-l|), standardised columns, beta* with k_true
    entries +-1 at seeded positions; least squares: y = X beta* + noise with
    sigma^2 = ||X beta*||^2 / (n SNR); logistic and squared hinge:
    P(y_i = +1) = sigmoid(x_i^T beta*).  Poisson and Gamma: columns of unit norm
    (the convention of the paper's real data), a log link with the linear
    predictor eta = 0.5 (X beta*) / std(X beta*), y ~ Poisson(e^eta) or
    y ~ Gamma(shape 2, mean e^eta) (the sum of two exponentials)."""
    if loss in (POISSON, GAMMA):
        P = make_problem(n, p, r=r, seed=seed, loss=LSQ, k_true=k_true, snr=snr, x_dtype=F64,
                         lambda2=lambda2, M=M, k=k)
        X = P.X / np.sqrt(n)
        xb = P.X @ P.beta_star
        eta = 0.5 * xb / max(float(np.std(xb)), 1e-300)
        mu = np.exp(eta)
        if loss == POISSON:
            y = _poisson(mu, uniform(seed, _S_COUNT, n))
        else:
            u = uniform(seed, _S_COUNT, 2 * n)
            y = 0.5 * mu * (-np.log1p(-u[:n]) - np.log1p(-u[n:]))
            y = np.maximum(y, 1e-300)
        if x_dtype == F32:
            X = X.astype(np.float32)
        elif x_dtype == BF16:
            X = f64_to_bf16(X)
        return Problem(X, y, P.beta_star, loss, float(lambda2), float(M), int(k), x_dtype,
                       dict(n=n, p=p, r=r, seed=seed, k_true=k_true, unit_norm=True))
    support = np.sort(_choose(seed, _S_SUPPORT, p, min(k_true, p)))
    signs = np.where(uniform(seed, _S_SIGN, support.size) < 0.5, -1.0, 1.0)
    beta_star = np.zeros(p)
    beta_star[support] = signs
    dt = {F64: np.float64, F32: np.float32, BF16: np.uint16}[x_dtype]
    X = np.empty((n, p), dtype=dt)
    xb = np.zeros(n)
    rc = _L().ksg_make_X(n, p, float(r), int(seed), _DT_CODE[x_dtype], X.ctypes.data,
                         beta_star.ctypes.data_as(C.POINTER(C.c_double)),
                         xb.ctypes.data_as(C.POINTER(C.c_double)), _threads())
    if rc != 0:
        raise RuntimeError(f"ksg_make_X failed ({rc})")
    if loss == LSQ:
        sigma = np.sqrt(float(xb @ xb) / (n * snr))
        y = xb + sigma * normal(seed, _S_NOISE, n)
    else:
        prob = 1.0 / (1.0 + np.exp(-xb))
        y = np.where(uniform(seed, _S_LABEL, n) < prob, 1.0, -1.0)
    return Problem(X, y, beta_star, loss, float(lambda2), float(M), int(k), x_dtype,
                   dict(n=n, p=p, r=r, seed=seed, k_true=k_true, snr=snr))


def quantize_fp8(X):
    """FP8 e4m3 storage of a matrix with one power-of-two scale per column:
    s_j = 2^ceil(log2(max_i |X_ij| / 448)), bits = e4m3(X / s) (round to nearest
    even).  Returns (uint8 bits, float32 scales); the represented matrix is
    fp8_values(bits) * s, exact in FP32."""
    import torch
    Xf = np.asarray(X, dtype=np.float32)
    amax = np.abs(Xf).max(axis=0)
    e = np.ceil(np.log2(np.maximum(amax, 1e-30) / 448.0)).astype(np.int32)
    e = np.clip(e, -100, 100)
    s = np.ldexp(np.float32(1.0), e).astype(np.float32)
    q = torch.from_numpy(Xf / s).to(torch.float8_e4m3fn)
    return q.view(torch.uint8).numpy().copy(), s


def fp8_values(bits):
    """The e4m3 values of FP8 bits (exact in float32)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(bits)).view(torch.float8_e4m3fn).to(torch.float32).numpy()


def node_sets(p, count, *, seed=0, max_zero=200, max_one=9):
    """Seeded branch-and-bound nodes: |S0| ~ U{0..max_zero}, |S1| ~ U{0..max_one},
    disjoint, positions uniform.  Returns a list of (S0, S1) int32 arrays."""
    u = uniform(seed, _S_NODES, 2 * count)
    out = []
    for b in range(count):
        nz = min(int(u[2 * b] * (max_zero + 1)), p)
        no = min(int(u[2 * b + 1] * (max_one + 1)), p - nz)
        idx = _choose(seed, _S_NODES, p, nz + no, salt=b + 1)
        out.append((np.sort(idx[:nz]).astype(np.int32), np.sort(idx[nz:]).astype(np.int32)))
    return out


def warm_perturbation(p, count, *, seed=0, var=1e-2):
    """N(0, var) perturbations (count x p) for warm starts."""
    return np.sqrt(var) * normal(seed, _S_WARM, count * p).reshape(count, p)


# --------------------------------------------------------------------------
# Device-side generation (large serving problems)

def device_problem(n, p, *, r=0.5, seed=0, loss=LSQ, k_true=5, snr=5.0, device="cuda", block=256):
    """The ``make_problem`` recipe drawn on a CUDA device with torch's generator:
    the same distribution (AR(1) Toeplitz rows, standardised columns, BF16 X,
    +-1 ground truth at seeded positions, the same label rules), not the same
    numbers.  Used where host generation of multi-GB matrices would dominate.
    The AR(1) recursion runs over blocks of ``block`` columns: inside a block the
    columns are x_{j0+t} = r^{t+1} x_{j0-1} + sum_{l<=t} s r^{t-l} e_{j0+l}
    (s = sqrt(1 - r^2)), one small product per block.
    Returns (X as an n x p torch.bfloat16 device tensor, y float64, beta*)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    support = np.sort(_choose(seed, _S_SUPPORT, p, min(k_true, p)))
    signs = np.where(uniform(seed, _S_SIGN, support.size) < 0.5, -1.0, 1.0)
    beta_star = np.zeros(p)
    beta_star[support] = signs
    s = float(np.sqrt(1.0 - r * r))
    t = torch.arange(block, device=device, dtype=torch.float64)
    d = t[None, :] - t[:, None]
    T = torch.where(d >= 0, s * torch.pow(torch.tensor(float(r), dtype=torch.float64, device=device),
                                             d.clamp(min=0)), torch.zeros_like(d)).float()
    rpow = torch.pow(torch.tensor(float(r), dtype=torch.float64, device=device), t + 1).float()
    X = torch.empty((n, p), dtype=torch.bfloat16, device=device)
    prev = torch.zeros(n, device=device)
    xb = torch.zeros(n, dtype=torch.float64, device=device)
    for j0 in range(0, p, block):
        w = min(block, p - j0)
        E = torch.randn((n, w), generator=g, device=device)
        if j0 == 0:
            E[:, 0] /= s           # x_0 = e_0
        raw = prev[:, None] * rpow[None, :w] + E @ T[:w, :w]
        prev = raw[:, w - 1].clone()
        mu = raw.mean(0, keepdim=True)
        sd = (raw - mu).pow(2).mean(0, keepdim=True).sqrt()
        X[:, j0:j0 + w] = ((raw - mu) / sd).to(torch.bfloat16)
        sel = support[(support >= j0) & (support < j0 + w)]
        for j in sel:
            xb += beta_star[j] * X[:, int(j)].double()
    xb_h = xb.cpu().numpy()
    if loss == LSQ:
        sigma = np.sqrt(float(xb_h @ xb_h) / (n * snr))
        y = xb_h + sigma * torch.randn(n, generator=g, device=device, dtype=torch.float64).cpu().numpy()
    else:
        prob = 1.0 / (1.0 + np.exp(-xb_h))
        y = np.where(torch.rand(n, generator=g, device=device, dtype=torch.float64).cpu().numpy() < prob,
                     1.0, -1.0)
    return X, y, beta_star


def serving_mix(count, *, seed=0):
    """Problem parameters of the serving stream: least squares or logistic,
    n ~ U{2000..40000}, p ~ U{1000..100000}, k ~ U{5..50},
    lambda2 in {1e-3, 1e-2, 1e-1}, M ~ U[1, 5], Toeplitz r in {0.1, 0.5, 0.9}."""
    u = uniform(seed, _S_MIX, 8 * count)
    out = []
    for i in range(count):
        v = u[8 * i:8 * i + 8]
        out.append(dict(loss=LSQ if v[0] < 0.5 else LOGISTIC,
                        n=2000 + int(v[1] * 38001), p=1000 + int(v[2] * 99001),
                        k=5 + int(v[3] * 46), lambda2=(1e-3, 1e-2, 1e-1)[min(int(v[4] * 3), 2)],
                        M=1.0 + 4.0 * float(v[5]), r=(0.1, 0.5, 0.9)[min(int(v[6] * 3), 2)],
                        seed=int(v[7] * 2**31)))
    return out


def poisson_arrivals(rate, duration, *, seed=0):
    """Arrival times (seconds) of a Poisson stream of the given rate over [0, duration)."""
    m = int(rate * duration * 3 + 64)
    gaps = -np.log(np.maximum(uniform(seed, _S_ARRIVAL, m), 1e-300)) / rate
    t = np.cumsum(gaps)
    return t[t < duration]


# --------------------------------------------------------------------------
# Named workloads (sizes and parameters of the benchmark configurations)

def cfg_small_lsq(seed=0):
    """Least squares, FP64, n=500, p=100, k=5, lambda2=1, M=2, Toeplitz 0.5, 5 x +-1, SNR 5."""
    return make_problem(500, 100, r=0.5, seed=seed, loss=LSQ, k_true=5, snr=5.0, x_dtype=F64,
                        lambda2=1.0, M=2.0, k=5)


def cfg_single_node_f32(seed=0, n=20000, p=50000):
    """Least squares, FP32, n=20000, p=50000, k=20, lambda2=0.1, M=1.5, Toeplitz 0.9, 20 x +-1."""
    return make_problem(n, p, r=0.9, seed=seed, loss=LSQ, k_true=20, snr=5.0, x_dtype=F32,
                        lambda2=0.1, M=1.5, k=20)


def cfg_batched_logistic(seed=0, n=10000, p=5000):
    """Logistic, BF16, n=10000, p=5000, k=10, lambda2=0.01, M=3, Toeplitz 0.5, 10 x +-1."""
    return make_problem(n, p, r=0.5, seed=seed, loss=LOGISTIC, k_true=10, x_dtype=BF16,
                        lambda2=0.01, M=3.0, k=10)
