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


def _hop_distances_from_A(dims, src):
    """Hop distance of every site from `src` by breadth-first search over the
    site graph of the dense matrix A (sites coupled by a nonzero 12 x 12 block)."""
    A = dense(dims, "haar", 1, 0.12)
    V = int(np.prod(dims))
    blocks = np.abs(A).reshape(V, 12, V, 12).max(axis=(1, 3)) > 0
    dist = np.full(V, -1)
    dist[src] = 0
    frontier = [src]
    while frontier:
        nxt = []
        for s in frontier:
            for r in np.nonzero(blocks[s])[0]:
                if dist[r] < 0:
                    dist[r] = dist[s] + 1
                    nxt.append(r)
        frontier = nxt
    return dist


def test_torus_distance_is_the_hop_distance_of_A():
    dims = (4, 2, 3, 4)
    for src in (0, 7, 53):
        ref = _hop_distances_from_A(dims, src)
        got = [M.torus_distance(dims, src, r) for r in range(int(np.prod(dims)))]
        assert np.array_equal(ref, got), src


def test_distance_colouring_probing_is_exact_up_to_its_distance():
    """A distance-4 colouring makes probing exact for degrees 1..4 and, since
    same-coloured sites 5 hops apart exist, not for degree 5 (Sec. 3.1: p_3 of
    degree 4 probed with a distance-4 colouring of the graph of A)."""
    dims = (4, 4, 4, 4)
    op = operator(dims, "haar", 1, 0.12)
    A = dense(dims, "haar", 1, 0.12)
    colours, nc = M.distance_colouring(dims, 4)
    V = int(np.prod(dims))
    assert nc < V // 2
    for deg in (1, 4):
        roots = np.linspace(0.8, 1.3, deg + 1) + 0.1j
        got = M.probing_trace_colours(op, {"kind": "single", "roots": roots}, colours, nc)
        assert abs(got - _exact_trace(A, roots)) < 1e-10 * abs(got), deg
    roots = np.linspace(0.8, 1.3, 6) + 0.1j
    got = M.probing_trace_colours(op, {"kind": "single", "roots": roots}, colours, nc)
    assert abs(got - _exact_trace(A, roots)) > 1e-6 * abs(got)


def test_colour_table_probing_reduces_to_the_period_colouring():
    dims = (4, 2, 2, 4)
    op = operator(dims, "haar", 3, 0.12)
    spec = {"kind": "composite", "inner": np.array([1.1 + 0.1j, 0.8]), "outer": np.array([0.9, 1.3 + 0.2j])}
    t, z, y, x = np.meshgrid(*[np.arange(L) for L in dims[::-1]], indexing="ij")
    colours = ((x % 2) + 2 * (y % 2) + 4 * (z % 2) + 8 * (t % 2)).reshape(-1)
    a = M.probing_trace_colours(op, spec, colours, 16)
    b = M.probing_trace(op, spec, 2)
    assert abs(a - b) < 1e-13 * abs(b)
