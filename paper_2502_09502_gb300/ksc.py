"""ctypes binding of the C ABI declared in ``include/ksc.h``.

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libksc.so``.  There is no fallback -- importing this module raises if
the library has not been built (``python -m paper_2502_09502_gb300.build``).
The functions keep the C names (``ksc_problem_create``, ``ksc_solve_node`` ...);
``Problem`` and ``Node`` are small conveniences over them.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libksc.so")

KSC_OK, KSC_ERR_INVALID_ARG, KSC_ERR_OOM, KSC_ERR_ADMISSION = 0, 1, 2, 3
KSC_ERR_INFEASIBLE_NODE, KSC_NOT_CONVERGED, KSC_ERR_TIMEOUT = 4, 5, 6
KSC_ERR_CUDA, KSC_ERR_UNIMPLEMENTED = 7, 8
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "oom", 3: "admission", 4: "infeasible_node",
                5: "not_converged", 6: "timeout", 7: "cuda", 8: "unimplemented"}
KSC_LOSS_LSQ, KSC_LOSS_LOGISTIC, KSC_LOSS_SQHINGE, KSC_LOSS_POISSON, KSC_LOSS_GAMMA = 0, 1, 2, 3, 4
KSC_F64, KSC_F32, KSC_BF16, KSC_FP8 = 0, 1, 2, 3   # KSC_FP8: e4m3 with power-of-two column scales
KSC_E4M3_PIECES = 5                                 # E4M3 pieces per vector row (ksc_tc_gemm_e4m3)
KSC_FLAG_RESTART_OFF, KSC_FLAG_MOMENTUM_OFF, KSC_FLAG_EIG = 1, 2, 4
KSC_KERNEL_GRADIENT, KSC_KERNEL_PROX, KSC_KERNEL_FORWARD = 0, 1, 2
KSC_KERNEL_B_RESID, KSC_KERNEL_B_GRAD, KSC_KERNEL_B_PROX, KSC_KERNEL_B_FWD, KSC_KERNEL_B_STEP = (
    3, 4, 5, 6, 7)
KSC_KERNEL_B_CERT, KSC_KERNEL_B_ANCHOR = 8, 9
KSC_KERNEL_PROX_SELECT, KSC_KERNEL_PROX_APPLY = 10, 11

# every symbol include/ksc.h declares
EXPORTS = ["ksc_problem_create", "ksc_problem_destroy", "ksc_problem_bytes", "ksc_problem_info",
           "ksc_solve_node", "ksc_solve_batch", "ksc_bnb_solve", "ksc_prox_g", "ksc_g_value", "ksc_gstar",
           "ksc_prox_g_noalloc", "ksc_prox_g_batch", "ksc_problem_profile", "ksc_problem_kernel_time",
           "ksc_problem_launch_count", "ksc_problem_solve_stats", "ksc_tc_gemm", "ksc_tc_gemm_sk", "ksc_tc_gemm_e4m3", "ksc_g_value_batch",
           "ksc_tc_exact",
           "ksc_server_create", "ksc_server_submit", "ksc_server_poll", "ksc_server_latency",
           "ksc_server_stats", "ksc_server_destroy", "ksc_problem_batch_node_state", "ksc_problem_eig_lambda",
           "ksc_problem_set_eig_lambda",
           "ksc_last_error", "ksc_version"]


class KscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ProblemDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int64), ("x_dtype", C.c_int), ("X", C.c_void_p),
                ("ldx", C.c_int64), ("y", C.POINTER(C.c_double)), ("loss", C.c_int),
                ("x_on_device", C.c_int32), ("lipschitz", C.c_double), ("col_scale", C.POINTER(C.c_float))]


class NodeC(C.Structure):
    _fields_ = [("lambda2", C.c_double), ("M", C.c_double), ("k", C.c_int32),
                ("fixed_zero", C.POINTER(C.c_int32)), ("n_zero", C.c_int32),
                ("fixed_one", C.POINTER(C.c_int32)), ("n_one", C.c_int32),
                ("warm_beta", C.POINTER(C.c_double)), ("incumbent", C.c_double),
                ("rel_gap_tol", C.c_double), ("max_iter", C.c_int32), ("flags", C.c_uint32)]


class ResultC(C.Structure):
    _fields_ = [("beta", C.POINTER(C.c_double)), ("z", C.POINTER(C.c_double)),
                ("primal", C.c_double), ("dual_bound", C.c_double), ("rel_gap", C.c_double),
                ("iters", C.c_int32), ("restarts", C.c_int32), ("pruned", C.c_int32),
                ("status", C.c_int)]


class BnbParams(C.Structure):
    _fields_ = [("lambda2", C.c_double), ("M", C.c_double), ("k", C.c_int32), ("opt_gap", C.c_double),
                ("max_nodes", C.c_int64), ("time_limit_s", C.c_double), ("batch", C.c_int32),
                ("node_rel_gap", C.c_double), ("node_max_iter", C.c_int32), ("node_flags", C.c_uint32)]


class BnbResultC(C.Structure):
    _fields_ = [("beta", C.POINTER(C.c_double)), ("incumbent", C.c_double), ("lower_bound", C.c_double),
                ("gap", C.c_double), ("nodes", C.c_int64), ("pruned", C.c_int64), ("closed", C.c_int64),
                ("heuristic_solves", C.c_int64), ("replays", C.c_int64), ("max_open", C.c_int64),
                ("seconds", C.c_double), ("certified", C.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -m paper_2502_09502_gb300.build)")
    L = C.CDLL(LIB_PATH)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    L.ksc_problem_create.argtypes = [C.POINTER(ProblemDesc), C.c_void_p, C.POINTER(C.c_void_p)]
    L.ksc_problem_destroy.argtypes = [C.c_void_p]
    L.ksc_problem_bytes.argtypes = [C.c_void_p]
    L.ksc_problem_bytes.restype = C.c_size_t
    L.ksc_problem_info.argtypes = [C.c_void_p, dp, ip]
    L.ksc_solve_node.argtypes = [C.c_void_p, C.POINTER(NodeC), C.POINTER(ResultC), C.c_void_p]
    L.ksc_solve_batch.argtypes = [C.c_void_p, C.POINTER(NodeC), C.c_int32, C.POINTER(ResultC),
                                  C.c_void_p]
    L.ksc_bnb_solve.argtypes = [C.c_void_p, C.POINTER(BnbParams), C.POINTER(BnbResultC), C.c_void_p]
    L.ksc_prox_g.argtypes = [dp, C.c_int64, C.c_int32, C.c_double, C.c_double, dp, ip]
    L.ksc_g_value.argtypes = [dp, C.c_int64, C.c_int32, C.c_double, dp, dp]
    L.ksc_gstar.argtypes = [dp, C.c_int64, C.c_int32, C.c_double, dp]
    L.ksc_problem_profile.argtypes = [C.c_void_p, C.c_int32]
    L.ksc_problem_kernel_time.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int64), dp,
                                          C.c_int32]
    L.ksc_problem_launch_count.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
    L.ksc_problem_solve_stats.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.c_int32]
    L.ksc_prox_g_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_double,
                                     C.c_void_p, C.c_void_p, C.c_void_p]
    L.ksc_prox_g_batch.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                   C.c_int32, C.c_double, C.c_double, C.c_void_p]
    L.ksc_g_value_batch.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_double,
                                    C.c_void_p, C.c_void_p]
    L.ksc_tc_gemm.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                              C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_int64, C.c_int32,
                              C.c_void_p]
    L.ksc_tc_gemm_sk.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int64,
                                 C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_int64, C.c_int32,
                                 C.c_int32, C.c_void_p]
    L.ksc_tc_gemm_e4m3.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_int32,
                                   C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                                   C.c_void_p]
    L.ksc_tc_exact.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_int32, C.c_int64,
                               C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.c_void_p]
    L.ksc_server_create.argtypes = [C.c_size_t, C.c_int32, C.POINTER(C.c_void_p)]
    L.ksc_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(NodeC), C.POINTER(C.c_uint64)]
    L.ksc_server_poll.argtypes = [C.c_void_p, C.c_uint64, C.POINTER(ResultC), C.c_int32]
    L.ksc_server_latency.argtypes = [C.c_void_p, C.c_uint64, dp]
    L.ksc_server_stats.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_int32]
    L.ksc_server_destroy.argtypes = [C.c_void_p]
    L.ksc_problem_batch_node_state.argtypes = [C.c_void_p, C.c_int32, dp, C.c_int32]
    L.ksc_problem_eig_lambda.argtypes = [C.c_void_p, C.c_void_p, dp]
    L.ksc_problem_set_eig_lambda.argtypes = [C.c_void_p, C.c_void_p, C.c_double]
    L.ksc_last_error.restype = C.c_char_p
    L.ksc_version.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("ksc_problem_bytes", "ksc_last_error", "ksc_version"):
            getattr(L, name).restype = C.c_int   # ksc_status
    return L


lib = _load()


def ksc_last_error() -> str:
    return lib.ksc_last_error().decode()


def ksc_version() -> str:
    return lib.ksc_version().decode()


def _check(st, allowed=(KSC_OK,)):
    if st not in allowed:
        raise KscError(st, ksc_last_error())
    return st


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)  # torch.cuda.Stream


# ---------------------------------------------------------------- C names

def ksc_problem_create(desc: ProblemDesc, stream=None):
    h = C.c_void_p()
    _check(lib.ksc_problem_create(C.byref(desc), _stream_ptr(stream), C.byref(h)))
    return h


def ksc_problem_destroy(h):
    return lib.ksc_problem_destroy(h)


def ksc_problem_bytes(h) -> int:
    return int(lib.ksc_problem_bytes(h))


def ksc_problem_info(h):
    L = C.c_double()
    it = C.c_int32()
    _check(lib.ksc_problem_info(h, C.byref(L), C.byref(it)))
    return L.value, it.value


def ksc_solve_node(h, node: NodeC, res: ResultC, stream=None):
    return lib.ksc_solve_node(h, C.byref(node), C.byref(res), _stream_ptr(stream))


def ksc_solve_batch(h, nodes, results, stream=None):
    return lib.ksc_solve_batch(h, nodes, len(nodes), results, _stream_ptr(stream))


def ksc_prox_g(w, k, M, rho, want_top=True):
    w = np.ascontiguousarray(w, dtype=np.float64)
    p = w.size
    out = np.zeros(p)
    q = min(int(k), p)
    top = np.full(max(q, 1), -1, dtype=np.int32)
    _check(lib.ksc_prox_g(_dptr(w), p, int(k), float(M), float(rho), _dptr(out),
                          top.ctypes.data_as(C.POINTER(C.c_int32)) if want_top else None))
    return out, top[:q]


def ksc_g_value(beta, k, M, want_z=True):
    b = np.ascontiguousarray(beta, dtype=np.float64)
    g = C.c_double()
    z = np.zeros(b.size)
    _check(lib.ksc_g_value(_dptr(b), b.size, int(k), float(M), C.byref(g),
                           _dptr(z) if want_z else None))
    return (g.value, z) if want_z else g.value


def ksc_gstar(a, k, M):
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = C.c_double()
    _check(lib.ksc_gstar(_dptr(a), a.size, int(k), float(M), C.byref(out)))
    return out.value


def ksc_prox_g_noalloc(w_ptr, p, k, M, rho, beta_ptr, top_ptr=None, stream=None):
    """Device-pointer prox without any device allocation (see include/ksc.h).
    Returns the ksc_status; the work is enqueued on `stream`."""
    return lib.ksc_prox_g_noalloc(C.c_void_p(w_ptr), int(p), int(k), float(M), float(rho),
                                  C.c_void_p(beta_ptr), C.c_void_p(top_ptr) if top_ptr else None,
                                  _stream_ptr(stream))


def ksc_prox_g_batch(w_ptr, ldw, beta_ptr, ldb, p, count, k, M, rho, stream=None):
    """Prox of g for `count` device rows at once (see include/ksc.h).  Returns the
    ksc_status; the work is enqueued on `stream`."""
    return lib.ksc_prox_g_batch(C.c_void_p(w_ptr), int(ldw), C.c_void_p(beta_ptr), int(ldb), int(p),
                                int(count), int(k), float(M), float(rho), _stream_ptr(stream))


def ksc_g_value_batch(beta_ptr, ldb, p, count, k, M, g_ptr, stream=None):
    """g of `count` device rows at once (see include/ksc.h).  Returns the ksc_status;
    the work is enqueued on `stream`."""
    return lib.ksc_g_value_batch(C.c_void_p(beta_ptr), int(ldb), int(p), int(count), int(k), float(M),
                                 C.c_void_p(g_ptr), _stream_ptr(stream))


def g_value_rows(B, k, M, stream=None):
    """B: 2-D float64 CUDA tensor (rows contiguous); returns g of every row (device)."""
    import torch
    assert B.is_cuda and B.dtype == torch.float64 and B.dim() == 2 and B.stride(1) == 1
    g = torch.empty(B.shape[0], dtype=torch.float64, device=B.device)
    _check(ksc_g_value_batch(B.data_ptr(), B.stride(0), B.shape[1], B.shape[0], k, M, g.data_ptr(), stream))
    return g


def prox_g_rows(W, k, M, rho, out=None, stream=None):
    """W: 2-D float64 CUDA tensor (rows contiguous); returns the prox of every row."""
    import torch
    assert W.is_cuda and W.dtype == torch.float64 and W.dim() == 2 and W.stride(1) == 1
    if out is None:
        out = torch.empty_like(W)
    _check(ksc_prox_g_batch(W.data_ptr(), W.stride(0), out.data_ptr(), out.stride(0), W.shape[1],
                            W.shape[0], k, M, rho, stream))
    return out


def ksc_tc_gemm(a_ptr, pieces, m, m_pad, k, lda, b_ptr, n, ldb, d_ptr, ldd, tile_n, stream=None):
    """Tensor-core product on device buffers (see include/ksc.h); blocks until done."""
    _check(lib.ksc_tc_gemm(C.c_void_p(a_ptr), int(pieces), int(m), int(m_pad), int(k), int(lda),
                           C.c_void_p(b_ptr), int(n), int(ldb), C.c_void_p(d_ptr), int(ldd),
                           int(tile_n), _stream_ptr(stream)))


def ksc_tc_exact(a_ptr, c, k, lda, v_ptr, r, ldv, d_ptr, ldd, stream=None) -> float:
    """Exact tensor-core product D = V A^T on device buffers (see include/ksc.h);
    blocks until done; returns the factor of its error bound."""
    eps = C.c_double(0.0)
    _check(lib.ksc_tc_exact(C.c_void_p(a_ptr), int(c), int(k), int(lda), C.c_void_p(v_ptr), int(r), int(ldv),
                            C.c_void_p(d_ptr), int(ldd), C.byref(eps), _stream_ptr(stream)))
    return eps.value


def ksc_tc_gemm_e4m3(a_ptr, m, m_pad, k, lda, b_ptr, n, ldb, rs_ptr, cs_ptr, d_ptr, ldd, tile_n, grid,
                     stream=None):
    """E4M3 tensor-core product on device buffers (see include/ksc.h); blocks until done."""
    _check(lib.ksc_tc_gemm_e4m3(C.c_void_p(a_ptr), int(m), int(m_pad), int(k), int(lda), C.c_void_p(b_ptr),
                                int(n), int(ldb), C.c_void_p(rs_ptr), C.c_void_p(cs_ptr) if cs_ptr else None,
                                C.c_void_p(d_ptr), int(ldd), int(tile_n), int(grid), _stream_ptr(stream)))


def ksc_tc_gemm_sk(a_ptr, pieces, m, m_pad, k, lda, b_ptr, n, ldb, d_ptr, ldd, tile_n, grid, stream=None):
    """Stream-K tensor-core product on device buffers (see include/ksc.h); blocks until done."""
    _check(lib.ksc_tc_gemm_sk(C.c_void_p(a_ptr), int(pieces), int(m), int(m_pad), int(k), int(lda),
                              C.c_void_p(b_ptr), int(n), int(ldb), C.c_void_p(d_ptr), int(ldd),
                              int(tile_n), int(grid), _stream_ptr(stream)))


def ksc_problem_profile(h, enable: bool):
    _check(lib.ksc_problem_profile(h, int(bool(enable))))


def ksc_problem_kernel_time(h, kernel, reset=False):
    n = C.c_int64()
    ms = C.c_double()
    _check(lib.ksc_problem_kernel_time(h, int(kernel), C.byref(n), C.byref(ms), int(bool(reset))))
    return n.value, ms.value


BATCH_NODE_STATE = ("tol_loop", "best_primal", "best_dual", "gap", "last_primal", "last_dual", "g",
                    "restarts", "iters", "cert_gap")


def ksc_problem_batch_node_state(h, index):
    buf = (C.c_double * len(BATCH_NODE_STATE))()
    _check(lib.ksc_problem_batch_node_state(h, int(index), buf, len(BATCH_NODE_STATE)))
    return dict(zip(BATCH_NODE_STATE, list(buf)))


def ksc_problem_eig_lambda(h, stream=None) -> float:
    lam = C.c_double()
    _check(lib.ksc_problem_eig_lambda(h, _stream_ptr(stream), C.byref(lam)))
    return lam.value


def ksc_problem_set_eig_lambda(h, lam, stream=None):
    _check(lib.ksc_problem_set_eig_lambda(h, _stream_ptr(stream), float(lam)))


def ksc_problem_launch_count(h) -> int:
    n = C.c_int64()
    _check(lib.ksc_problem_launch_count(h, C.byref(n)))
    return n.value


SOLVE_STATS = ("iters", "sparse_forward", "prox_fallback", "prox_predicted", "dual_predicted",
               "lanczos", "batch_certificates", "batch_anchors", "tile_fwd", "stream_k_fwd", "tile_grad",
               "stream_k_grad")


def ksc_problem_solve_stats(h):
    buf = (C.c_int32 * len(SOLVE_STATS))()
    _check(lib.ksc_problem_solve_stats(h, buf, len(SOLVE_STATS)))
    return dict(zip(SOLVE_STATS, list(buf)))


# ---------------------------------------------------------------- helpers

_DT = {np.dtype(np.float64): KSC_F64, np.dtype(np.float32): KSC_F32, np.dtype(np.uint16): KSC_BF16}


@dataclass
class Result:
    beta: np.ndarray | None
    z: np.ndarray | None
    primal: float
    dual_bound: float
    rel_gap: float
    iters: int
    restarts: int
    pruned: bool
    status: str


class Node:
    """A branch-and-bound node (fixed sets S0/S1) with its solve parameters."""

    def __init__(self, lambda2, M, k, fixed_zero=(), fixed_one=(), warm_beta=None,
                 incumbent=math.inf, rel_gap_tol=1e-6, max_iter=100000, flags=0):
        self.zero = np.ascontiguousarray(fixed_zero, dtype=np.int32)
        self.one = np.ascontiguousarray(fixed_one, dtype=np.int32)
        self.warm = None if warm_beta is None else np.ascontiguousarray(warm_beta, dtype=np.float64)
        self.c = NodeC(float(lambda2), float(M), int(k),
                       self.zero.ctypes.data_as(C.POINTER(C.c_int32)) if self.zero.size else None,
                       int(self.zero.size),
                       self.one.ctypes.data_as(C.POINTER(C.c_int32)) if self.one.size else None,
                       int(self.one.size),
                       _dptr(self.warm) if self.warm is not None else None,
                       float(incumbent), float(rel_gap_tol), int(max_iter), int(flags))


class Problem:
    """Owns a ksc_problem handle.  X: numpy array (copied to the device; bf16 as
    uint16 bits) or a CUDA torch tensor (borrowed: kept alive by this object)."""

    def __init__(self, X, y, loss=KSC_LOSS_LSQ, lipschitz=0.0, stream=None, x_dtype=None, col_scale=None):
        """col_scale: FP8 X only -- p power-of-two column scales (the matrix is X_ij s_j)."""
        self._keep = []
        y = np.ascontiguousarray(y, dtype=np.float64)
        if hasattr(X, "data_ptr"):  # torch tensor on the device
            import torch
            assert X.is_cuda and X.is_contiguous()
            code = {torch.float64: KSC_F64, torch.float32: KSC_F32, torch.bfloat16: KSC_BF16,
                    torch.float8_e4m3fn: KSC_FP8}[X.dtype]
            ptr, on_dev = X.data_ptr(), 1
            n, p = X.shape
            self._keep.append(X)
        else:
            X = np.ascontiguousarray(X)
            code = _DT[X.dtype] if x_dtype is None else x_dtype
            ptr, on_dev = X.ctypes.data, 0
            n, p = X.shape
            self._keep.append(X)
        self.n, self.p = int(n), int(p)
        self._keep.append(y)
        sc = None
        if code == KSC_FP8:
            if col_scale is None:
                raise ValueError("FP8 X needs col_scale")
            sc = np.ascontiguousarray(col_scale, dtype=np.float32)
            self._keep.append(sc)
        self.desc = ProblemDesc(self.n, self.p, code, ptr, self.p, _dptr(y), int(loss), on_dev,
                                float(lipschitz), sc.ctypes.data_as(C.POINTER(C.c_float)) if sc is not None else None)
        self.h = ksc_problem_create(self.desc, stream)
        self.stream = stream

    def close(self):
        if getattr(self, "h", None):
            ksc_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def L(self):
        return ksc_problem_info(self.h)[0]

    @property
    def power_iters(self):
        return ksc_problem_info(self.h)[1]

    @property
    def bytes(self):
        return ksc_problem_bytes(self.h)

    def solve(self, node: Node, want_beta=True, want_z=True, allow=(KSC_OK, KSC_NOT_CONVERGED,
                                                                      KSC_ERR_INFEASIBLE_NODE)):
        beta = np.zeros(self.p) if want_beta else None
        z = np.zeros(self.p) if want_z else None
        res = ResultC(_dptr(beta) if want_beta else None, _dptr(z) if want_z else None)
        st = ksc_solve_node(self.h, node.c, res, self.stream)
        _check(st, allow)
        return Result(beta, z, res.primal, res.dual_bound, res.rel_gap, res.iters, res.restarts,
                      bool(res.pruned), STATUS_NAMES[res.status if st == KSC_OK else st])

    def eig_lambda(self):
        """ksc_problem_eig_lambda: the certified shift of the eigen-perspective
        relaxation (a lower bound on lambda_min(X^T X))."""
        return ksc_problem_eig_lambda(self.h, self.stream)

    def set_eig_lambda(self, lam):
        """ksc_problem_set_eig_lambda: certify lam below lambda_min(X^T X) and use it."""
        ksc_problem_set_eig_lambda(self.h, lam, self.stream)

    def bnb(self, lambda2, M, k, opt_gap=1e-4, max_nodes=0, time_limit_s=0.0, batch=256,
            node_rel_gap=1e-6, node_max_iter=20000, node_flags=0):
        """ksc_bnb_solve: best-first branch and bound over the node relaxations.
        Returns (incumbent beta, dict of the result fields)."""
        prm = BnbParams(float(lambda2), float(M), int(k), float(opt_gap), int(max_nodes),
                        float(time_limit_s), int(batch), float(node_rel_gap), int(node_max_iter),
                        int(node_flags))
        beta = np.zeros(self.p)
        res = BnbResultC()
        res.beta = _dptr(beta)
        _check(lib.ksc_bnb_solve(self.h, C.byref(prm), C.byref(res), _stream_ptr(self.stream)))
        out = {name: getattr(res, name) for name, _ in BnbResultC._fields_ if name != "beta"}
        out["certified"] = bool(out["certified"])
        return beta, out

    def solve_batch(self, nodes, want_beta=True, want_z=False,
                    allow=(KSC_OK, KSC_NOT_CONVERGED, KSC_ERR_INFEASIBLE_NODE)):
        """ksc_solve_batch over a list of Node; returns one Result per node."""
        B = len(nodes)
        arr = (NodeC * B)(*[nd.c for nd in nodes])
        res = (ResultC * B)()
        betas = [np.zeros(self.p) if want_beta else None for _ in range(B)]
        zs = [np.zeros(self.p) if want_z else None for _ in range(B)]
        for i in range(B):
            res[i].beta = _dptr(betas[i]) if want_beta else None
            res[i].z = _dptr(zs[i]) if want_z else None
        st = lib.ksc_solve_batch(self.h, arr, B, res, _stream_ptr(self.stream))
        _check(st, allow)
        return [Result(betas[i], zs[i], res[i].primal, res[i].dual_bound, res[i].rel_gap,
                       res[i].iters, res[i].restarts, bool(res[i].pruned),
                       STATUS_NAMES[res[i].status]) for i in range(B)]


SERVER_STATS = ("completed", "replays", "sessions", "peak_bytes", "waited_for_budget",
                "admitted_while_running")


class Server:
    """ksc_server_*: continuous batching of node solves over resident problems."""

    def __init__(self, hbm_budget_bytes, max_slots=128):
        h = C.c_void_p()
        _check(lib.ksc_server_create(C.c_size_t(int(hbm_budget_bytes)), int(max_slots), C.byref(h)))
        self.h = h
        self._p = {}

    def submit(self, problem: "Problem", node: Node) -> int:
        t = C.c_uint64()
        _check(lib.ksc_server_submit(self.h, problem.h, C.byref(node.c), C.byref(t)))
        self._p[t.value] = problem.p
        return t.value

    def poll(self, ticket, timeout_ms=-1, want_beta=True, want_z=False,
             allow=(KSC_OK, KSC_NOT_CONVERGED, KSC_ERR_INFEASIBLE_NODE)):
        """Result of a request, or None when the wait expires."""
        p = self._p.get(ticket, 0)
        want_beta = want_beta and p > 0
        want_z = want_z and p > 0
        beta = np.zeros(p) if want_beta else None
        z = np.zeros(p) if want_z else None
        res = ResultC(_dptr(beta) if want_beta else None, _dptr(z) if want_z else None)
        st = lib.ksc_server_poll(self.h, C.c_uint64(ticket), C.byref(res), int(timeout_ms))
        if st == KSC_ERR_TIMEOUT and self._pending(ticket):
            return None
        self._p.pop(ticket, None)
        _check(st, allow)
        return Result(beta, z, res.primal, res.dual_bound, res.rel_gap, res.iters, res.restarts,
                      bool(res.pruned), STATUS_NAMES[res.status if st == KSC_OK else st])

    def _pending(self, ticket):
        # a timed-out poll leaves the ticket queued; a released one is unknown
        return ticket in self._p

    def latency(self, ticket) -> float:
        s = C.c_double()
        _check(lib.ksc_server_latency(self.h, C.c_uint64(ticket), C.byref(s)))
        return s.value

    def stats(self):
        arr = (C.c_int64 * len(SERVER_STATS))()
        _check(lib.ksc_server_stats(self.h, arr, len(SERVER_STATS)))
        return dict(zip(SERVER_STATS, list(arr)))

    def close(self):
        if getattr(self, "h", None):
            lib.ksc_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
