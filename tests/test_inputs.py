"""The seeded input generator: Philox4x32-10 known answers, determinism, statistics."""
import numpy as np

import ksc_inputs as G


def test_philox_known_answers():
    # Random123 known-answer vectors for Philox4x32-10 (Salmon et al., SC'11)
    assert G.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert G.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert G.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                           [0xA4093822, 0x299F31D0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_problem_is_deterministic_and_standardised():
    a = G.make_problem(300, 64, r=0.5, seed=3, k_true=4)
    b = G.make_problem(300, 64, r=0.5, seed=3, k_true=4)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.y, b.y)
    assert np.allclose(a.X.mean(0), 0, atol=1e-12)
    assert np.allclose((a.X ** 2).sum(0), 300, rtol=1e-12)
    assert np.count_nonzero(a.beta_star) == 4 and set(np.abs(a.beta_star[a.beta_star != 0])) == {1.0}


def test_dtypes_are_roundings_of_the_same_matrix():
    a = G.make_problem(50, 40, seed=1, x_dtype=G.F64)
    b = G.make_problem(50, 40, seed=1, x_dtype=G.F32)
    c = G.make_problem(50, 40, seed=1, x_dtype=G.BF16)
    assert np.array_equal(a.X.astype(np.float32), b.X)
    assert np.max(np.abs(c.X64() - a.X)) <= 2 ** -8 * np.abs(a.X).max()


def test_toeplitz_correlation():
    P = G.make_problem(4000, 12, r=0.7, seed=2, x_dtype=G.F64)
    C = np.corrcoef(P.X.T)
    for lag in (1, 2, 3):
        assert abs(np.mean(np.diag(C, lag)) - 0.7 ** lag) < 0.03


def test_labels_and_node_sets():
    P = G.make_problem(500, 30, seed=4, loss=G.LOGISTIC)
    assert set(np.unique(P.y)) == {-1.0, 1.0}
    nodes = G.node_sets(300, 50, seed=9)
    for s0, s1 in nodes:
        assert len(s0) <= 200 and len(s1) <= 9
        assert len(set(s0) & set(s1)) == 0
        assert len(set(s0)) == len(s0) and len(set(s1)) == len(s1)
    again = G.node_sets(300, 50, seed=9)
    assert all(np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
               for x, y in zip(nodes, again))


def test_squared_hinge_problems_share_the_classification_labels():
    a = G.make_problem(400, 30, seed=6, loss=G.LOGISTIC)
    b = G.make_problem(400, 30, seed=6, loss=G.SQHINGE)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.y, b.y)
    assert set(np.unique(b.y)) == {-1.0, 1.0}


def test_fp8_quantizer_scales_and_values():
    P = G.make_problem(200, 40, seed=7, x_dtype=G.F32)
    X = P.X.astype(np.float32)
    X[:, 3] *= 1e-3                                   # a column of another magnitude
    bits, s = G.quantize_fp8(X)
    assert bits.dtype == np.uint8 and bits.shape == X.shape and s.shape == (40,)
    m, e = np.frexp(s)
    assert np.all(m == 0.5)                           # powers of two
    v = G.fp8_values(bits)
    assert np.abs(v).max() <= 448.0
    rep = v.astype(np.float64) * s.astype(np.float64)
    # the represented matrix is exact in FP32 and within e4m3's half ulp of X
    assert np.array_equal(rep.astype(np.float32).astype(np.float64), rep)
    amax = np.abs(X).max(0)
    assert np.all(np.abs(rep - X) <= 2.0 ** -4 * np.abs(X) + 2.0 ** -9 * s)
    assert np.all(amax / s <= 448.0) and np.all(amax / s > 224.0 - 1e-3)   # the smallest fitting scale


def test_serving_mix_and_arrivals():
    mix = G.serving_mix(64, seed=3)
    assert mix == G.serving_mix(64, seed=3)
    for m in mix:
        assert m["loss"] in (G.LSQ, G.LOGISTIC)
        assert 2000 <= m["n"] <= 40000 and 1000 <= m["p"] <= 100000 and 5 <= m["k"] <= 50
        assert m["lambda2"] in (1e-3, 1e-2, 1e-1) and 1.0 <= m["M"] <= 5.0 and m["r"] in (0.1, 0.5, 0.9)
    t = G.poisson_arrivals(50.0, 40.0, seed=2)
    assert np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < 40.0
    assert abs(len(t) / 40.0 - 50.0) < 4 * np.sqrt(50.0 / 40.0) + 1     # Poisson count within 4 sigma
    assert np.array_equal(t, G.poisson_arrivals(50.0, 40.0, seed=2))


def test_count_responses_unit_norm_columns_and_label_ranges():
    # Poisson counts are non-negative integers, Gamma responses positive; both use
    # unit-norm columns; BF16 storage rounds the same matrix
    for loss in (G.POISSON, G.GAMMA):
        P = G.make_problem(300, 40, seed=4, loss=loss, k_true=3)
        assert np.allclose(np.linalg.norm(P.X, axis=0), 1.0, atol=1e-12)
        if loss == G.POISSON:
            assert np.all(P.y >= 0) and np.all(P.y == np.round(P.y)) and P.y.sum() > 0
        else:
            assert np.all(P.y > 0)
        Pb = G.make_problem(300, 40, seed=4, loss=loss, k_true=3, x_dtype=G.BF16)
        assert np.array_equal(Pb.y, P.y)
        assert np.max(np.abs(Pb.X64() - P.X)) <= 2.0 ** -8 * np.abs(P.X).max()
