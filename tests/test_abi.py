"""The C ABI library loads and exports every function include/ksc.h declares;
argument checks that return before any CUDA call work without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ksc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ksc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def ksc():
    import __graft_entry__ as g
    g.build()
    from paper_2502_09502_gb300 import ksc as K
    return K


def test_every_declared_symbol_is_exported(ksc):
    decl = _declared()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(ksc.lib, name), name
    assert set(decl) <= set(ksc.EXPORTS) | {"ksc_last_error", "ksc_version"}


def test_version_and_error_strings(ksc):
    assert "sm_103a" in ksc.ksc_version()
    assert isinstance(ksc.ksc_last_error(), str)


def test_invalid_arguments_are_rejected_before_cuda(ksc):
    out = C.c_void_p(123)
    assert ksc.lib.ksc_problem_create(None, None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert out.value is None
    y = np.zeros(3)
    d = ksc.ProblemDesc(0, 4, ksc.KSC_F64, 1, 4, y.ctypes.data_as(C.POINTER(C.c_double)), 0, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "n and p" in ksc.ksc_last_error()
    d = ksc.ProblemDesc(3, 4, 9, 1, 4, y.ctypes.data_as(C.POINTER(C.c_double)), 0, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    d = ksc.ProblemDesc(3, 4, ksc.KSC_F64, 1, 2, y.ctypes.data_as(C.POINTER(C.c_double)), 0, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "ldx" in ksc.ksc_last_error()
    yl = np.array([1.0, 0.5, -1.0])
    d = ksc.ProblemDesc(3, 4, ksc.KSC_F64, 1, 4, yl.ctypes.data_as(C.POINTER(C.c_double)),
                        ksc.KSC_LOSS_LOGISTIC, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "labels" in ksc.ksc_last_error()
    d = ksc.ProblemDesc(3, 4, ksc.KSC_F64, 1, 4, yl.ctypes.data_as(C.POINTER(C.c_double)),
                        ksc.KSC_LOSS_SQHINGE, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "labels" in ksc.ksc_last_error()
    d = ksc.ProblemDesc(3, 4, ksc.KSC_F64, 1, 4, y.ctypes.data_as(C.POINTER(C.c_double)), 5, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "loss" in ksc.ksc_last_error()
    # Poisson responses >= 0, Gamma responses > 0 (checked before any CUDA call)
    yneg = np.array([1.0, -2.0, 0.0])
    d = ksc.ProblemDesc(3, 4, ksc.KSC_F64, 1, 4, yneg.ctypes.data_as(C.POINTER(C.c_double)),
                        ksc.KSC_LOSS_POISSON, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "Poisson" in ksc.ksc_last_error()
    yzero = np.array([1.0, 0.5, 0.0])
    d = ksc.ProblemDesc(3, 4, ksc.KSC_F64, 1, 4, yzero.ctypes.data_as(C.POINTER(C.c_double)),
                        ksc.KSC_LOSS_GAMMA, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "Gamma" in ksc.ksc_last_error()
    # FP8 X: power-of-two column scales required (checked before any CUDA call)
    d = ksc.ProblemDesc(3, 4, ksc.KSC_FP8, 1, 4, y.ctypes.data_as(C.POINTER(C.c_double)), 0, 0, 0.0)
    assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "col_scale" in ksc.ksc_last_error()
    for bad in ([1.0, 0.75, 2.0, 4.0], [1.0, 2.0 ** -101, 1.0, 1.0], [1.0, -2.0, 1.0, 1.0]):
        sc = np.array(bad, dtype=np.float32)
        d = ksc.ProblemDesc(3, 4, ksc.KSC_FP8, 1, 4, y.ctypes.data_as(C.POINTER(C.c_double)), 0, 0, 0.0,
                            sc.ctypes.data_as(C.POINTER(C.c_float)))
        assert ksc.lib.ksc_problem_create(C.byref(d), None, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    w = np.ones(4)
    dp = C.POINTER(C.c_double)
    assert ksc.lib.ksc_prox_g(w.ctypes.data_as(dp), 4, 2, 1.0, -1.0, w.ctypes.data_as(dp),
                              None) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_prox_g(None, 4, 2, 1.0, 1.0, w.ctypes.data_as(dp), None) == \
        ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_prox_g(w.ctypes.data_as(dp), 0, 2, 1.0, 1.0, w.ctypes.data_as(dp),
                              None) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_g_value(w.ctypes.data_as(dp), 4, -1, 1.0, w.ctypes.data_as(dp), None) == \
        ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_gstar(w.ctypes.data_as(dp), 4, 1, 0.0, w.ctypes.data_as(dp)) == \
        ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_solve_node(None, None, None, None) == ksc.KSC_ERR_INVALID_ARG
    lam = C.c_double(-1.0)
    assert ksc.lib.ksc_problem_eig_lambda(None, None, C.byref(lam)) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_problem_set_eig_lambda(None, None, 1.0) == ksc.KSC_ERR_INVALID_ARG
    # batched prox on device rows: every argument check comes before any CUDA call
    fb = ksc.lib.ksc_prox_g_batch
    assert fb(None, 8, None, 8, 8, 3, 2, 1.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG   # NULL rows
    assert fb(None, 8, None, 8, 8, 0, 2, 1.0, 1.0, None) == ksc.KSC_OK                 # nothing to do
    assert fb(16, 8, 4096, 8, 0, 3, 2, 1.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG      # p = 0
    assert fb(16, 4, 4096, 8, 8, 3, 2, 1.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG      # ldw < p
    assert "ldw" in ksc.ksc_last_error()
    assert fb(16, 8, 4096, 8, 8, -3, 2, 1.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG     # count < 0
    assert fb(16, 8, 4096, 8, 8, 3, 2, 0.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG      # M <= 0
    assert fb(16, 8, 4096, 8, 8, 3, 2, 1.0, float("nan"), None) == ksc.KSC_ERR_INVALID_ARG
    assert fb(16, 4096, 1 << 20, 4096, 4096, 3, 2048, 1.0, 1.0, None) == ksc.KSC_ERR_UNIMPLEMENTED
    assert fb(4096, 8, 4096 + 64, 8, 8, 3, 2, 1.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG   # overlap
    assert "overlap" in ksc.ksc_last_error()
    # leading dimensions whose byte spans would overflow int64 are refused before
    # the overlap test
    assert fb(16, 1 << 61, 1 << 40, 8, 8, 3, 2, 1.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG
    assert "too large" in ksc.ksc_last_error()
    assert fb(16, 8, 1 << 40, 1 << 61, 8, 3, 2, 1.0, 1.0, None) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_problem_info(None, None, None) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_problem_bytes(None) == 0
    assert ksc.lib.ksc_problem_destroy(None) == ksc.KSC_OK


def test_struct_layouts_match_header(ksc):
    # offsets the C compiler uses for the ABI structs (x86-64 and aarch64 LP64)
    assert C.sizeof(ksc.ProblemDesc) == 72
    assert ksc.ProblemDesc.X.offset == 24 and ksc.ProblemDesc.lipschitz.offset == 56
    assert ksc.ProblemDesc.col_scale.offset == 64
    assert C.sizeof(ksc.NodeC) == 88
    assert ksc.NodeC.warm_beta.offset == 56 and ksc.NodeC.flags.offset == 84
    assert C.sizeof(ksc.ResultC) == 56
    assert ksc.ResultC.status.offset == 52
    assert C.sizeof(ksc.BnbParams) == 72
    assert ksc.BnbParams.opt_gap.offset == 24 and ksc.BnbParams.node_max_iter.offset == 64
    assert ksc.BnbParams.node_flags.offset == 68
    assert C.sizeof(ksc.BnbResultC) == 96
    assert ksc.BnbResultC.seconds.offset == 80 and ksc.BnbResultC.certified.offset == 88


def test_bnb_arguments_are_rejected_before_cuda(ksc):
    prm = ksc.BnbParams(0.1, 1.0, 3, 1e-4, 0, 0.0, 64, 1e-6, 1000)
    res = ksc.BnbResultC()
    f = ksc.lib.ksc_bnb_solve
    assert f(None, C.byref(prm), C.byref(res), None) == ksc.KSC_ERR_INVALID_ARG
    bad = ksc.BnbParams(0.1, 1.0, 3, 1e-4, 0, 0.0, 0, 1e-6, 1000)          # batch 0
    assert f(C.c_void_p(8), C.byref(bad), C.byref(res), None) == ksc.KSC_ERR_INVALID_ARG
    bad = ksc.BnbParams(-0.1, 1.0, 3, 1e-4, 0, 0.0, 64, 1e-6, 1000)        # lambda2 < 0
    assert f(C.c_void_p(8), C.byref(bad), C.byref(res), None) == ksc.KSC_ERR_INVALID_ARG
    bad = ksc.BnbParams(0.1, 1.0, 4096, 1e-4, 0, 0.0, 64, 1e-6, 1000)      # k beyond capacity
    assert f(C.c_void_p(8), C.byref(bad), C.byref(res), None) == ksc.KSC_ERR_UNIMPLEMENTED


def test_server_arguments_are_rejected_before_cuda(ksc):
    out = C.c_void_p(7)
    assert ksc.lib.ksc_server_create(C.c_size_t(0), 16, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert out.value is None
    assert ksc.lib.ksc_server_create(C.c_size_t(1 << 30), 0, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_server_create(C.c_size_t(1 << 30), 2000, C.byref(out)) == ksc.KSC_ERR_INVALID_ARG
    assert "max_slots" in ksc.ksc_last_error()
    t = C.c_uint64()
    assert ksc.lib.ksc_server_submit(None, None, None, C.byref(t)) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_server_poll(None, 1, None, 0) == ksc.KSC_ERR_INVALID_ARG
    assert ksc.lib.ksc_server_destroy(None) == ksc.KSC_OK
    st = (C.c_int64 * 6)()
    assert ksc.lib.ksc_server_stats(None, st, 6) == ksc.KSC_ERR_INVALID_ARG


def test_header_constants_match_the_binding(ksc):
    # every KSC_* enumerator and #define of include/ksc.h has the same value in
    # the Python binding (a drift would pass wrong codes through the ABI)
    src = open(os.path.join(ROOT, "include", "ksc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    consts = {}
    for name, val in re.findall(r"\b(KSC_[A-Z0-9_]+)\s*=\s*(\d+)", src):
        consts[name] = int(val)
    for name, val in re.findall(r"#define\s+(KSC_[A-Z0-9_]+)\s+(0x[0-9a-fA-F]+u?|\d+u?)", src):
        consts[name] = int(val.rstrip("u"), 0)
    assert len(consts) >= 20
    alias = {"KSC_FP8_E4M3_COLSCALE": "KSC_FP8"}
    for name, val in consts.items():
        py = alias.get(name, name)
        assert hasattr(ksc, py), name
        assert getattr(ksc, py) == val, (name, getattr(ksc, py), val)
