"""Pins of the oracle's polynomials: GMRES identity, power basis, dense spectra."""

import itertools
import json
import os

import numpy as np
import pytest

from conftest import dense, operator
from oracle import krylov as K
from oracle import polynomial as P
from paper_2306_09559_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


@pytest.mark.parametrize("m", [5, 12, 41])
def test_gmres_identity(m):
    # The GMRES iterate x_m (x_0 = 0) equals p(A) b with p's roots the harmonic
    # Ritz values at step m (Sec. 3.1: pi = 1 - alpha p is the residual polynomial)
    op = operator((4, 4, 4, 4), "haar", 0, 0.12)
    b = synth.random_unit_vector(op.n, 100)
    V, Hbar, beta = K.arnoldi(op, b, m)
    x_gm, res = K.gmres_iterate(V, Hbar, beta, m)
    th = K.harmonic_ritz(Hbar, m)
    x_pf = P.apply_poly(op, th[P.leja_order(th)], b)
    assert np.linalg.norm(x_pf - x_gm) < 1e-10 * np.linalg.norm(x_gm)
    assert abs(np.linalg.norm(b - op(x_pf)) - res) < 1e-10


def test_power_basis_agrees_at_low_degree():
    op = operator((2, 2, 2, 4), "haar", 1, 0.12)
    b = synth.random_unit_vector(op.n, 3)
    for m in (1, 2, 6, 12):
        V, Hbar, beta = K.arnoldi(op, b, m)
        th = K.harmonic_ritz(Hbar, m)
        pf = P.apply_poly(op, th, b)
        pb = P.apply_poly_power_basis(op, P.poly_coefficients(th), b)
        assert np.linalg.norm(pf - pb) < 1e-10 * np.linalg.norm(pf)


def test_root_order_invariance_low_degree(rng):
    op = operator((2, 2, 2, 2), "haar", 2, 0.12)
    b = synth.random_unit_vector(op.n, 4)
    V, Hbar, beta = K.arnoldi(op, b, 8)
    th = K.harmonic_ritz(Hbar, 8)
    ref = P.apply_poly(op, th, b)
    for _ in range(3):
        perm = rng.permutation(th.size)
        assert np.linalg.norm(P.apply_poly(op, th[perm], b) - ref) < 1e-11 * np.linalg.norm(ref)


def test_scalar_values_on_a_diagonal_matrix(rng):
    d = rng.uniform(0.3, 2.0, 50) + 1j * rng.uniform(-0.5, 0.5, 50)
    roots = rng.uniform(0.5, 2.0, 7) + 1j * rng.uniform(-0.3, 0.3, 7)
    v = rng.standard_normal(50) + 0j
    y = P.apply_poly(lambda w: d * w if w.ndim == 1 else d[:, None] * w, roots, v)
    assert np.allclose(y, P.poly_value(roots, d) * v, rtol=1e-13, atol=0)
    # 1 - lambda p(lambda) = pi(lambda), and pi vanishes at its roots
    assert np.allclose(1 - d * P.poly_value(roots, d), P.residual_poly_value(roots, d), atol=1e-12)
    assert np.max(np.abs(P.residual_poly_value(roots, roots))) < 1e-14


def test_dense_trace_of_poly():
    # Tr p(A) = sum_i p(lambda_i) over the dense spectrum
    A = dense((2, 2, 2, 2), "haar", 0, 0.12)
    op = operator((2, 2, 2, 2), "haar", 0, 0.12)
    b = synth.random_unit_vector(op.n, 8)
    V, Hbar, beta = K.arnoldi(op, b, 10)
    th = K.harmonic_ritz(Hbar, 10)
    PA = P.apply_poly(lambda X: A @ X, th, np.eye(op.n, dtype=complex))
    lam = np.linalg.eigvals(A)
    assert abs(np.trace(PA) - np.sum(P.poly_value(th, lam))) < 1e-10 * op.n


def test_composite_equals_spectral_product():
    # p_1(A) = p_in(A) p_out(A p_in(A)) through the eigendecomposition of A
    dims = (2, 2, 2, 2)
    A = dense(dims, "haar", 0, 0.12)
    op = operator(dims, "haar", 0, 0.12)
    b = synth.random_unit_vector(op.n, 9)
    inner = K.gmres_polynomials(op, b, [4])[0]
    outer, m_out, _ = K.pp_gmres_roots(op, inner, b, m_out=6)
    lam, S = np.linalg.eig(A)
    ref = S @ (P.composite_value(inner, outer, lam) * np.linalg.solve(S, b))
    got = P.apply_composite(op, inner, outer, b)
    assert np.linalg.norm(got - ref) < 1e-9 * np.linalg.norm(ref)


def test_composite_degree_and_matvec_count():
    for m_in, m_out, deg in GOLDEN["composite_degrees"]["cases"]:
        assert P.composite_degree(m_in, m_out) == deg
        assert P.matvecs_composite(m_in, m_out) == deg
    op = operator((2, 2, 2, 2), "haar", 0, 0.12)
    b = synth.random_unit_vector(op.n, 1)
    for m_in, m_out in ((3, 4), (1, 5), (5, 1)):
        inner = np.linspace(0.5, 1.5, m_in) + 0.1j
        outer = np.linspace(0.6, 1.4, m_out) - 0.05j
        op.matvecs = 0
        P.apply_composite(op, inner, outer, b)
        assert op.matvecs == m_in * m_out - 1
    for m in (1, 2, 9):
        op.matvecs = 0
        P.apply_poly(op, np.linspace(0.5, 1.5, m), b)
        assert op.matvecs == m - 1


def test_leja_order_by_definition(rng):
    for trial in range(5):
        r = rng.standard_normal(9) + 1j * rng.standard_normal(9)
        order = P.leja_order(r)
        assert sorted(order.tolist()) == list(range(9))
        assert order[0] == np.argmax(np.abs(r))
        for k in range(1, 9):
            rest = [i for i in range(9) if i not in order[:k]]
            prods = [np.prod(np.abs(r[i] - r[order[:k]])) for i in rest]
            assert rest[int(np.argmax(prods))] == order[k]


def test_orthogonalisation_cost_arithmetic():
    # Sec. 3.2 counts about m^2 vector operations for m Arnoldi steps
    for ms, cost in GOLDEN["orthogonalisation_cost"]["cases"]:
        assert sum(m * m for m in ms) == cost
