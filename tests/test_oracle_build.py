"""The all-cores build of the oracle (OpenMP over the rows of X v and over blocks
of columns of X^T r) is only a faster way to run the same arithmetic: every output
element is summed in the same order, so its results equal the single-threaded
build's bit for bit.  The benchmark's CPU baseline times it on every host core."""
import numpy as np

import ksc_inputs as G
from oracle import oracle as O


def test_openmp_build_gives_identical_results():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((700, 530))
    v, r = rng.standard_normal(530), rng.standard_normal(700)
    import ctypes as C
    dp = C.POINTER(C.c_double)
    L1 = O.lib(False)
    Lm = O.lib(True)
    for L in (L1, Lm):
        u = np.zeros(700)
        g = np.zeros(530)
        L.kso_matvec(X.ctypes.data, 0, 700, 530, 530, v.ctypes.data_as(dp), u.ctypes.data_as(dp))
        L.kso_rmatvec(X.ctypes.data, 0, 700, 530, 530, r.ctypes.data_as(dp), g.ctypes.data_as(dp))
        if L is L1:
            u1, g1 = u, g
    assert np.array_equal(u, u1) and np.array_equal(g, g1)
    P = G.make_problem(300, 120, r=0.5, seed=3, loss=G.LOGISTIC, k_true=4, x_dtype=G.F64,
                       lambda2=0.5, M=2.0, k=4)
    a = O.solve(P.X, P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-9)
    b = O.solve(P.X, P.y, P.loss, P.lambda2, P.M, P.k, tol=1e-9, openmp=True)
    assert a.iters == b.iters and a.dual == b.dual and np.array_equal(a.beta, b.beta)
    assert O.threads(False) == 1 and O.threads(True) >= 1
