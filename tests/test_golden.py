"""Hand-derived closed-form cases (tests/golden/closed_form_cases.txt) against the oracle."""
import os

import numpy as np
import pytest

from oracle import oracle as O

_PATH = os.path.join(os.path.dirname(__file__), "golden", "closed_form_cases.txt")


def _cases():
    out = []
    for line in open(_PATH):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        out.append([f.strip() for f in line.split("|")])
    return out


def _vec(s):
    return np.array([float(t) for t in s.split()])


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0] + ":" + c[1])
def test_closed_form_case(case):
    kind = case[0]
    if kind == "prox_g":
        w, k, rho, M, exp = _vec(case[1]), int(case[2]), float(case[3]), float(case[4]), _vec(case[5])
        got, _ = O.prox_g(w, k, rho, M)
    elif kind == "g":
        got = O.g_value(_vec(case[1]), int(case[2]), float(case[3]))
        exp = float(case[4])
    elif kind == "gstar":
        got = O.gstar(_vec(case[1]), int(case[2]), float(case[3]))
        exp = float(case[4])
    elif kind == "huber":
        got = O.huber(float(case[1]), float(case[2]))
        exp = float(case[3])
    elif kind == "negconj":
        got = O.neg_conj(int(case[1]), _vec(case[2]), _vec(case[3]))
        exp = float(case[4])
    elif kind == "loss":
        got = O.loss(int(case[1]), _vec(case[2]), _vec(case[3]))
        exp = float(case[4])
    elif kind == "eigbound":
        n, p = (int(t) for t in case[2].split())
        X = _vec(case[1]).reshape(n, p)
        got = O.dual_bound(X, _vec(case[3]), 0, float(case[4]), float(case[5]), int(case[6]), _vec(case[8]),
                           eig=float(case[7]))
        exp = float(case[9])
    else:
        raise AssertionError(kind)
    assert np.allclose(got, exp, rtol=1e-14, atol=1e-14), (got, exp)
