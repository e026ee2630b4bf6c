"""Pins of the oracle's Z4 noise: uniformity, independence, Hutchinson moments.

The exact Philox bit pattern is "parity unpinned" (no known-answer vector
offline); GPU and oracle are compared bit for bit in the GPU tests.
"""

import numpy as np

from oracle import philox


def test_symbol_frequencies_uniform():
    # 4 symbols x 12 entries x 2^18 sites ~ 3.1e6 draws per stream; 4 sigma
    q = philox.z4_symbols(seed=2024, level=1, noise_index=0, nsites=1 << 18).ravel()
    counts = np.bincount(q, minlength=4)
    n = q.size
    sigma = np.sqrt(n * 0.25 * 0.75)
    assert np.all(np.abs(counts - n / 4) < 4 * sigma)


def test_pair_independence_chi_square():
    q = philox.z4_symbols(seed=7, level=0, noise_index=3, nsites=1 << 16)
    # adjacent entries in a site, and the same entry at adjacent sites
    for a, b in ((q[:, :-1].ravel(), q[:, 1:].ravel()), (q[:-1, 0], q[1:, 0])):
        joint = np.bincount(4 * a + b, minlength=16)
        exp = a.size / 16
        chi2 = np.sum((joint - exp) ** 2 / exp)
        assert chi2 < 45.0   # 15 dof; p ~ 1e-4


def test_streams_differ_by_every_counter_word():
    base = philox.z4_symbols(1, 0, 0, 4096)
    for args in ((2, 0, 0), (1, 1, 0), (1, 0, 1)):
        other = philox.z4_symbols(args[0], args[1], args[2], 4096)
        # independent streams agree in ~1/4 of the entries
        assert 0.2 < np.mean(base == other) < 0.3
    hi = philox.z4_symbols(1 + (1 << 32), 0, 0, 4096)
    assert 0.2 < np.mean(base == hi) < 0.3


def test_values_and_mapping():
    b = philox.z4_noise(5, 2, 9, 64)
    assert set(np.round(b, 12)) <= {1, -1, 1j, -1j}
    q = philox.z4_symbols(5, 2, 9, 64).ravel()
    assert np.array_equal(b, np.array([1, 1j, -1, -1j])[q])


def test_hutchinson_second_moments():
    # E[b b^H] = I and E[b b^T] = 0 for Z4 noise: sample means over 4000 vectors
    nsites, N = 2, 4000
    B = philox.z4_block(11, 0, 0, N, nsites)
    bbH = B @ B.conj().T / N
    bbT = B @ B.T / N
    tol = 4 / np.sqrt(N)
    assert np.max(np.abs(bbH - np.eye(24))) < tol
    assert np.max(np.abs(bbT)) < tol
    assert np.allclose(np.diag(bbH), 1.0)
