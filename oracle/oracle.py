"""Python access to the FP64 CPU oracle (``ksc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use this module; the CUDA library never does.  It compiles
``ksc_oracle.c`` with gcc into ``oracle/_build/libksc_oracle.so`` on first use
(or when ``build()`` is called) and wraps each routine for numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ksc_oracle.c")
_HDR = os.path.join(_HERE, "ksc_oracle.h")
_OUT = os.path.join(_HERE, "_build", "libksc_oracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "libksc_oracle_omp.so")

LOSS_LSQ, LOSS_LOGISTIC, LOSS_SQHINGE, LOSS_POISSON, LOSS_GAMMA = 0, 1, 2, 3, 4
FREE, ZERO, ONE = 0, 1, 2
STATUS = {0: "converged", 1: "max_iter", 2: "pruned", 3: "primal_below", 4: "infeasible"}

_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle (plain C, -O2, no FP contraction so that x86 and Arm agree).
    openmp=True: the all-cores build (-fopenmp), identical results, used only to
    time the CPU baseline on every host core."""
    out = _OUT_OMP if openmp else _OUT
    stale = not os.path.exists(out) or any(
        os.path.getmtime(s) > os.path.getmtime(out) for s in (_SRC, _HDR))
    if force or stale:
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared"]
                              + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


_lib_omp = None


def lib(openmp: bool = False):
    """The single-threaded oracle library (default) or its all-cores build."""
    global _lib, _lib_omp
    if openmp:
        if _lib_omp is None:
            _lib_omp = C.CDLL(build(openmp=True))
            _declare(_lib_omp)
        return _lib_omp
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


def threads(openmp: bool = False) -> int:
    """Threads the oracle's matrix-vector products run on."""
    return int(lib(openmp).kso_threads())


_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_i8p = C.POINTER(C.c_int8)


class SolveArgs(C.Structure):
    _fields_ = [("X", C.c_void_p), ("x_dtype", C.c_int32), ("n", C.c_int64), ("p", C.c_int64),
                ("ldx", C.c_int64), ("y", _dp), ("loss", C.c_int32), ("lambda2", C.c_double),
                ("M", C.c_double), ("k", C.c_int64), ("state", _i8p), ("warm", _dp),
                ("L", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int64),
                ("restart", C.c_int32), ("momentum", C.c_int32), ("incumbent", C.c_double),
                ("eig", C.c_double)]


class SolveOut(C.Structure):
    _fields_ = [("primal", C.c_double), ("dual", C.c_double), ("gap", C.c_double),
                ("L", C.c_double), ("iters", C.c_int64), ("restarts", C.c_int64),
                ("status", C.c_int32)]


def _declare(L):
    L.kso_threads.restype = C.c_int
    L.kso_threads.argtypes = []
    L.kso_huber.restype = C.c_double
    L.kso_huber.argtypes = [C.c_double, C.c_double]
    L.kso_huber_prox.restype = C.c_double
    L.kso_huber_prox.argtypes = [C.c_double, C.c_double, C.c_double]
    L.kso_prox_gstar.argtypes = [_dp, C.c_int64, C.c_int64, C.c_double, C.c_double, _dp, _i64p]
    L.kso_prox_g.argtypes = [_dp, C.c_int64, C.c_int64, C.c_double, C.c_double, _dp, _i64p]
    L.kso_g_value.restype = C.c_double
    L.kso_g_value.argtypes = [_dp, C.c_int64, C.c_int64, C.c_double, _dp]
    L.kso_gstar.restype = C.c_double
    L.kso_gstar.argtypes = [_dp, C.c_int64, C.c_int64, C.c_double]
    L.kso_prox_g_node.argtypes = [_dp, C.c_int64, _i8p, C.c_int64, C.c_double, C.c_double,
                                  _dp, _i64p]
    L.kso_g_node.restype = C.c_double
    L.kso_g_node.argtypes = [_dp, C.c_int64, _i8p, C.c_int64, C.c_double, _dp]
    L.kso_Gstar_node.restype = C.c_double
    L.kso_Gstar_node.argtypes = [_dp, C.c_int64, _i8p, C.c_int64, C.c_double, C.c_double]
    L.kso_loss.restype = C.c_double
    L.kso_loss.argtypes = [C.c_int, _dp, _dp, C.c_int64]
    L.kso_loss_grad.argtypes = [C.c_int, _dp, _dp, C.c_int64, _dp]
    L.kso_neg_conj.restype = C.c_double
    L.kso_neg_conj.argtypes = [C.c_int, _dp, _dp, C.c_int64]
    L.kso_matvec.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_int64, _dp, _dp]
    L.kso_rmatvec.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_int64, _dp, _dp]
    L.kso_power_iteration.restype = C.c_double
    L.kso_power_iteration.argtypes = [C.c_void_p, C.c_int, C.c_int64, C.c_int64, C.c_int64,
                                      C.c_double, C.c_int64, _i64p]
    L.kso_solve.argtypes = [C.POINTER(SolveArgs), _dp, _dp, _dp, C.POINTER(SolveOut)]
    L.kso_dual_bound.restype = C.c_double
    L.kso_dual_bound.argtypes = [C.POINTER(SolveArgs), _dp]
    L.kso_primal.restype = C.c_double
    L.kso_primal.argtypes = [C.POINTER(SolveArgs), _dp]


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _state(state, p):
    if state is None:
        return None, None
    s = np.ascontiguousarray(state, dtype=np.int8)
    assert s.shape == (p,)
    return s, s.ctypes.data_as(_i8p)


def huber(a, M):
    return lib().kso_huber(float(a), float(M))


def huber_prox(x, c, M):
    return lib().kso_huber_prox(float(x), float(c), float(M))


def prox_gstar(mu, k, rho, M):
    mu, pm = _d(mu)
    p = mu.size
    al = np.zeros(p)
    perm = np.zeros(p, dtype=np.int64)
    lib().kso_prox_gstar(pm, p, int(k), float(rho), float(M), al.ctypes.data_as(_dp),
                         perm.ctypes.data_as(_i64p))
    return al, perm


def prox_g(w, k, rho, M):
    w, pw = _d(w)
    p = w.size
    b = np.zeros(p)
    perm = np.zeros(p, dtype=np.int64)
    lib().kso_prox_g(pw, p, int(k), float(rho), float(M), b.ctypes.data_as(_dp),
                     perm.ctypes.data_as(_i64p))
    return b, perm


def g_value(beta, k, M, want_z=False):
    beta, pb = _d(beta)
    z = np.zeros(beta.size)
    g = lib().kso_g_value(pb, beta.size, int(k), float(M), z.ctypes.data_as(_dp))
    return (g, z) if want_z else g


def gstar(a, k, M):
    a, pa = _d(a)
    return lib().kso_gstar(pa, a.size, int(k), float(M))


def prox_g_node(w, state, k, rho, M):
    w, pw = _d(w)
    p = w.size
    s, ps = _state(state, p)
    nfree = p if s is None else int((s == FREE).sum())
    kp = int(k) - (0 if s is None else int((s == ONE).sum()))
    b = np.zeros(p)
    top = np.full(max(1, min(max(kp, 0), nfree)), -1, dtype=np.int64)
    rc = lib().kso_prox_g_node(pw, p, ps, int(k), float(rho), float(M), b.ctypes.data_as(_dp),
                               top.ctypes.data_as(_i64p))
    if rc != 0:
        raise ValueError("infeasible node: |S1| > k")
    return b, top[:max(0, min(kp, nfree))]


def g_node(beta, state, k, M, want_z=False):
    beta, pb = _d(beta)
    s, ps = _state(state, beta.size)
    z = np.zeros(beta.size)
    g = lib().kso_g_node(pb, beta.size, ps, int(k), float(M), z.ctypes.data_as(_dp))
    return (g, z) if want_z else g


def Gstar_node(a, state, k, lambda2, M):
    a, pa = _d(a)
    s, ps = _state(state, a.size)
    return lib().kso_Gstar_node(pa, a.size, ps, int(k), float(lambda2), float(M))


def loss(kind, u, y):
    u, pu = _d(u)
    y, py = _d(y)
    return lib().kso_loss(int(kind), pu, py, u.size)


def loss_grad(kind, u, y):
    u, pu = _d(u)
    y, py = _d(y)
    g = np.zeros(u.size)
    lib().kso_loss_grad(int(kind), pu, py, u.size, g.ctypes.data_as(_dp))
    return g


def neg_conj(kind, zeta, y):
    z, pz = _d(zeta)
    y, py = _d(y)
    return lib().kso_neg_conj(int(kind), pz, py, z.size)


def _xptr(X):
    if X.dtype == np.float32:
        X = np.ascontiguousarray(X)
        return X, 1
    X = np.ascontiguousarray(X, dtype=np.float64)
    return X, 0


def matvec(X, v):
    X, dt = _xptr(X)
    v, pv = _d(v)
    out = np.zeros(X.shape[0])
    lib().kso_matvec(X.ctypes.data, dt, X.shape[0], X.shape[1], X.shape[1], pv,
                     out.ctypes.data_as(_dp))
    return out


def rmatvec(X, r):
    X, dt = _xptr(X)
    r, pr = _d(r)
    out = np.zeros(X.shape[1])
    lib().kso_rmatvec(X.ctypes.data, dt, X.shape[0], X.shape[1], X.shape[1], pr,
                      out.ctypes.data_as(_dp))
    return out


def power_iteration(X, tol=1e-10, max_iter=10000, openmp=False):
    X, dt = _xptr(X)
    it = C.c_int64(0)
    lam = lib(openmp).kso_power_iteration(X.ctypes.data, dt, X.shape[0], X.shape[1], X.shape[1],
                                    float(tol), int(max_iter), C.byref(it))
    return lam, it.value


@dataclass
class SolveResult:
    beta: np.ndarray
    z: np.ndarray
    primal: float
    dual: float
    gap: float
    L: float
    iters: int
    restarts: int
    status: str
    trace: np.ndarray | None = None


class _Args:
    """Keeps the numpy buffers alive while the C struct points at them."""

    def __init__(self, X, y, loss_kind, lambda2, M, k, state=None, warm=None, L=0.0,
                 tol=1e-12, max_iter=100000, restart=True, momentum=True,
                 incumbent=float("inf"), eig=0.0):
        if eig and loss_kind != 0:
            raise ValueError("the eigen-perspective relaxation is for least squares")
        self.X, dt = _xptr(X)
        n, p = self.X.shape
        self.y, py = _d(y)
        assert self.y.shape == (n,)
        self.state, ps = _state(state, p)
        if warm is not None:
            self.warm, pwm = _d(warm)
            assert self.warm.shape == (p,)
        else:
            self.warm, pwm = None, None
        self.c = SolveArgs(self.X.ctypes.data, dt, n, p, p, py, int(loss_kind), float(lambda2),
                           float(M), int(k), ps, pwm, float(L), float(tol), int(max_iter),
                           int(bool(restart)), int(bool(momentum)), float(incumbent), float(eig))
        self.n, self.p = n, p


def solve(X, y, loss_kind, lambda2, M, k, state=None, warm=None, L=0.0, tol=1e-12,
          max_iter=100000, restart=True, momentum=True, incumbent=float("inf"),
          want_trace=False, eig=0.0, openmp=False):
    """Restarted FISTA (Algorithm 3) on the node problem, in FP64; eig > 0: the
    eigen-perspective relaxation of App. D.2 with Q = X^T X - eig I."""
    a = _Args(X, y, loss_kind, lambda2, M, k, state, warm, L, tol, max_iter, restart,
              momentum, incumbent, eig)
    beta = np.zeros(a.p)
    z = np.zeros(a.p)
    trace = np.zeros(2 * max_iter) if want_trace else None
    out = SolveOut()
    lib(openmp).kso_solve(C.byref(a.c), beta.ctypes.data_as(_dp), z.ctypes.data_as(_dp),
                    trace.ctypes.data_as(_dp) if want_trace else None, C.byref(out))
    tr = trace[:2 * out.iters].reshape(-1, 2) if want_trace else None
    return SolveResult(beta, z, out.primal, out.dual, out.gap, out.L, out.iters, out.restarts,
                       STATUS[out.status], tr)


def dual_bound(X, y, loss_kind, lambda2, M, k, beta, state=None, eig=0.0):
    a = _Args(X, y, loss_kind, lambda2, M, k, state, eig=eig)
    b, pb = _d(beta)
    return lib().kso_dual_bound(C.byref(a.c), pb)


def primal(X, y, loss_kind, lambda2, M, k, beta, state=None, eig=0.0):
    a = _Args(X, y, loss_kind, lambda2, M, k, state, eig=eig)
    b, pb = _d(beta)
    return lib().kso_primal(C.byref(a.c), pb)


def lambda_min(X):
    """lambda_min(X^T X) (App. D.2) by a dense symmetric eigensolver in FP64
    (numpy's LAPACK routine as the step), clipped at 0."""
    X = np.asarray(X, dtype=np.float64)
    return max(0.0, float(np.linalg.eigvalsh(X.T @ X)[0]))
