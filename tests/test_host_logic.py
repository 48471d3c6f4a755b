"""Host-side planning rules of the single-node path, compiled on the CPU.

Two rules decide launch shapes and the Lipschitz constant without touching the
GPU: the rows per CTA of the streaming passes over X (whole waves of resident
CTAs) and the stop test of the Lanczos iteration for L (the step constant that
Algorithm 3 takes as input).  Both are inline host functions of the launch
header; a small harness built with the host compiler evaluates them here.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import ksc_inputs as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_09502_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

HARNESS = r"""
#include "ksc_launch.h"
#include <cstdio>
int main() {
  char op;
  while (std::scanf(" %c", &op) == 1) {
    if (op == 'R') {
      int rows, strips, slots;
      if (std::scanf("%d %d %d", &rows, &strips, &slots) != 3) return 1;
      std::printf("%d\n", ksc::balanced_rows(rows, strips, slots));
    } else {
      double t, p1, p2;
      if (std::scanf("%lf %lf %lf", &t, &p1, &p2) != 3) return 1;
      std::printf("%d\n", ksc::lanczos_stop(t, p1, p2) ? 1 : 0);
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    d = tmp_path_factory.mktemp("host_logic")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CUDA_INC, "-I", CSRC, str(src), "-o", str(exe)],
                   check=True, capture_output=True)

    def run(lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split()
        return [int(x) for x in out]
    return run


def rows_of(harness, cases):
    return harness([f"R {r} {s} {k}" for r, s, k in cases])


def stop_of(harness, triples):
    return [bool(x) for x in harness([f"S {float(t)!r} {float(a)!r} {float(b)!r}" for t, a, b in triples])]


def test_balanced_rows_known_shapes(harness):
    # 20000 x 50000 FP32 (49 strips of 1024 columns) on 152 SMs: 6 resident CTAs give
    # 93 row blocks of 216 rows = 4557 CTAs <= 5 x 912, five full waves; 5 per SM the
    # same 216 (4557 <= 6 x 760).  8000 x 20000 (20 strips) fits one wave: 45 blocks of
    # 180 rows (900 <= 912), or 38 of 212 (760 <= 760).
    got = rows_of(harness, [(20000, 49, 912), (20000, 49, 760), (8000, 20, 912), (8000, 20, 760)])
    assert got == [216, 216, 180, 212]
    # the last wave is full: 4557 of 5 x 912 slots, 900 of 912
    assert math.ceil(20000 / 216) * 49 / (5 * 912) > 0.99 and math.ceil(8000 / 180) * 20 / 912 > 0.98


def test_balanced_rows_minimises_waves_times_rows(harness):
    rng = np.random.default_rng(11)
    cases = [(int(rng.integers(1, 200001)), int(rng.integers(1, 401)), int(152 * rng.integers(1, 17)))
             for _ in range(300)]
    cases += [(1, 1, 152), (128, 1, 152), (257, 3, 152), (10**6, 1, 152)]
    got = rows_of(harness, cases)
    cost = lambda rows, strips, slots, r: math.ceil(math.ceil(rows / r) * strips / slots) * r
    for (rows, strips, slots), r in zip(cases, got):
        assert 128 <= r <= 256 and r % 4 == 0
        best = min(cost(rows, strips, slots, c) for c in range(128, 257, 4))
        assert cost(rows, strips, slots, r) == best
        # the largest of the equally good choices: fewest CTAs and partial sums
        assert all(cost(rows, strips, slots, c) > best for c in range(r + 4, 257, 4))


def test_lanczos_stop_cases(harness):
    lam = 1000.0
    # the first checks never stop
    assert stop_of(harness, [(900.0, -1.0, -1.0), (990.0, 900.0, -1.0)]) == [False, False]
    # a block that moves theta by at most 1e-5 of itself stops, either sign
    assert stop_of(harness, [(lam, lam * (1 - 9e-6), -1.0), (lam, lam * (1 + 9e-6), lam)]) == [True, True]
    # geometric convergence theta_k = lam (1 - c q^k): the Aitken tail is exact, so the
    # rule stops exactly when what is left is at most 1e-3 of theta
    for q in (0.2, 0.5, 0.8, 0.95):
        for c in (0.5, 0.05):
            th = [lam * (1 - c * q ** k) for k in range(200)]
            for k in range(2, 200):
                s = stop_of(harness, [(th[k], th[k - 1], th[k - 2])])[0]
                left = (lam - th[k]) / th[k]
                assert s == (left <= 1e-3 * (1 + 1e-9) or th[k] - th[k - 1] <= 1e-5 * th[k]), (q, c, k)
                if s:
                    assert left <= 1.001e-3
                    break
            else:
                pytest.fail("no stop")
    # rises that do not shrink (d2 >= d1) or a first rise that is not positive: no
    # extrapolation, only the 1e-5 test
    assert stop_of(harness, [(lam, lam - 2.0, lam - 3.0), (lam, lam - 1.0, lam - 1.0)]) == [False, False]


def _lanczos_thetas(X, steps):
    """Plain Lanczos on X^T X in FP64 from the library's start vector: the largest
    Ritz value after each step."""
    p = X.shape[1]
    j = np.arange(p, dtype=np.uint64)
    v = 1.0 + ((j + np.uint64(1)) * np.uint64(2654435761) % np.uint64(1000)).astype(np.float64) / 1000.0
    v /= np.linalg.norm(v)
    vprev, beta = np.zeros(p), 0.0
    al, be, th = [], [], []
    for _ in range(steps):
        w = X.T @ (X @ v)
        a = float(w @ v)
        w = w - a * v - beta * vprev
        b = float(np.linalg.norm(w))
        al.append(a)
        be.append(b)
        T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
        th.append(np.linalg.eigvalsh(T)[-1])
        vprev, v, beta = v, w / b, b
    return th


def test_lanczos_stop_on_the_single_node_spectrum(harness):
    # the single-node workload's design (Toeplitz 0.9, p > n: a continuum at the top of
    # the spectrum, where Lanczos converges slowest) at a tenth of its size
    P = G.make_problem(2000, 5000, r=0.9, seed=0, x_dtype=G.F32, k_true=20)
    X = P.X.astype(np.float64)
    lam = np.linalg.eigvalsh(X @ X.T)[-1]
    th = _lanczos_thetas(X, 96)
    checks = list(range(8, 97, 8))
    stop_at = old_at = None
    for i, m in enumerate(checks):
        t = th[m - 1]
        prev = th[checks[i - 1] - 1] if i >= 1 else -1.0
        prev2 = th[checks[i - 2] - 1] if i >= 2 else -1.0
        if stop_at is None and stop_of(harness, [(t, prev, prev2)])[0]:
            stop_at = m
        if old_at is None and prev > 0 and abs(t - prev) <= 1e-5 * t:
            old_at = m
    assert stop_at is not None and old_at is not None
    assert stop_at <= old_at
    t = th[stop_at - 1]
    # a lower estimate, within a fifth of L's 1% margin
    assert lam * (1 - 2e-3) <= t <= lam * (1 + 1e-12)
