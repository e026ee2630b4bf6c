"""Pins of the probing estimate (the exact trace of the lowest-degree level,
paper Sec. 5, step 3c, with a period-m distance colouring): with m equal to
the lattice extent every probe vector is a unit vector and the estimate is
the exact trace for any polynomial; for m > degree it is exact as well, since
p(A) couples only sites fewer than `degree + 1` hops apart; and it differs
from the exact trace when the degree reaches m."""

import numpy as np

from conftest import dense, operator
from oracle import mpmc as M


def _exact_trace(A, roots):
    # tr p(A) with p(A) = sum_i theta_i^{-1} prod_{j<i} (I - A/theta_j), from the dense matrix
    n = A.shape[0]
    P = np.zeros_like(A)
    W = np.eye(n, dtype=np.complex128)
    for th in roots:
        P += W / th
        W = W - (A @ W) / th
    return np.trace(P)


def test_probing_with_period_equal_to_extent_is_the_exact_trace():
    dims = (2, 2, 2, 2)
    op = operator(dims, "haar", 3, 0.13)
    roots = np.array([1.3 + 0.2j, 0.8 - 0.1j, 1.1 + 0.05j, 0.9 + 0.3j, 1.6])
    got = M.probing_trace(op, {"kind": "single", "roots": roots}, 2)
    ref = _exact_trace(dense(dims, "haar", 3, 0.13), roots)
    assert abs(got - ref) < 1e-11 * abs(ref)


def test_probing_is_exact_below_the_period():
    dims = (4, 4, 4, 4)
    op = operator(dims, "haar", 1, 0.12)
    A = dense(dims, "haar", 1, 0.12)
    for deg in (1, 2):              # degree of p: nroots - 1
        roots = np.linspace(0.8, 1.3, deg + 1) + 0.1j
        got = M.probing_trace(op, {"kind": "single", "roots": roots}, 4 if deg < 4 else 8)
        assert abs(got - _exact_trace(A, roots)) < 1e-10 * abs(got), deg
    roots = np.linspace(0.8, 1.3, 3) + 0.1j        # degree 2 < m = 4 but period 2 is too short
    got2 = M.probing_trace(op, {"kind": "single", "roots": roots}, 2)
    assert abs(got2 - _exact_trace(A, roots)) > 1e-6 * abs(got2)


def test_probe_vectors_partition_the_identity():
    dims = (4, 2, 2, 4)
    V = M.probing_vectors(dims, 2, list(range(12 * 16)))
    assert np.array_equal(V.sum(axis=1), np.ones(12 * 64))
    assert np.array_equal(V.T @ V, np.diag(np.full(12 * 16, 4.0)))
