"""Pins of the oracle's Krylov setup: Arnoldi, harmonic Ritz, PP-GMRES, eigen selection."""

import json
import os

import numpy as np

from conftest import dense, operator
from oracle import krylov as K
from oracle import polynomial as P
from paper_2306_09559_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_constants_from_the_paper():
    assert K.IMAGLIM == GOLDEN["deflation_constants"]["imaglim"]
    assert K.EVECTOL == GOLDEN["deflation_constants"]["evectol"]


def test_arnoldi_relation():
    op = operator((4, 4, 4, 4), "haar", 0, 0.12)
    b = synth.random_unit_vector(op.n, 1)
    m = 30
    V, H, beta = K.arnoldi(op, b, m)
    assert np.max(np.abs(op(V[:, :m]) - V @ H)) < 1e-12
    assert np.max(np.abs(V.conj().T @ V - np.eye(m + 1))) < 1e-13
    assert np.allclose(np.tril(H, -2), 0)


def test_harmonic_ritz_full_space_gives_eigenvalues(rng):
    # on a full Krylov space the harmonic Ritz values are the eigenvalues
    n = 40
    A = rng.standard_normal((n, n)) + 21 * np.eye(n)     # Example 1 construction, small n
    b = rng.standard_normal(n) + 0j
    V, H, beta = K.arnoldi(lambda v: A @ v, b, n)
    # h_{n+1,n} = 0 up to rounding: the standard-form correction vanishes
    th = K.harmonic_ritz(np.vstack([H[:n, :n], np.zeros((1, n))]), n)
    ev = np.linalg.eigvals(A)
    # every eigenvalue is matched by a distinct harmonic Ritz value
    dist = np.abs(th[:, None] - ev[None, :])
    assert np.max(np.min(dist, axis=0)) < 1e-8 and np.max(np.min(dist, axis=1)) < 1e-8
    assert len(set(np.argmin(dist, axis=1))) == n


def test_harmonic_ritz_values_are_residual_polynomial_roots():
    # the GMRES residual b - A x_m vanishes in no direction except through pi(A) b;
    # check pi(A) b = b - A x_m with pi built from the harmonic Ritz values
    op = operator((2, 2, 2, 4), "haar", 3, 0.13)
    b = synth.random_unit_vector(op.n, 2)
    m = 15
    V, H, beta = K.arnoldi(op, b, m)
    x, res = K.gmres_iterate(V, H, beta, m)
    th = K.harmonic_ritz(H, m)
    r = P.apply_residual_poly(op, th[P.leja_order(th)], b)
    assert np.linalg.norm(r - (b - op(x))) < 1e-10


def test_pp_gmres_identity():
    # p_out from GMRES on B = A p_in(A): its iterate equals p_out(B) b
    op = operator((4, 4, 4, 4), "haar", 0, 0.12)
    b = synth.random_unit_vector(op.n, 5)
    inner = K.gmres_polynomials(op, b, [6])[0]
    B = K.pp_operator(op, inner)
    m = 9
    V, H, beta = K.arnoldi(B, b, m)
    x, _ = K.gmres_iterate(V, H, beta, m)
    outer, m_out, rel = K.pp_gmres_roots(op, inner, b, m_out=m)
    assert m_out == m
    assert np.linalg.norm(P.apply_poly(B, outer, b) - x) < 1e-10 * np.linalg.norm(x)
    # with a tolerance, the chosen step is the first one below it
    outer2, m2, rel2 = K.pp_gmres_roots(op, inner, b, rtol=1e-3, max_m=60)
    hist = K.gmres_residual_history(K.arnoldi(B, b, m2)[1], 1.0)
    assert rel2 < 1e-3 and (m2 == 1 or hist[m2 - 2] >= 1e-3)


def test_pp_arnoldi_eigenpairs_and_selection():
    dims, kappa = (2, 2, 2, 4), 0.14
    op = operator(dims, "haar", 1, kappa)
    A = dense(dims, "haar", 1, kappa)
    b = synth.random_unit_vector(op.n, 6)
    inner = K.gmres_polynomials(op, b, [5])[0]
    lam, Z = K.pp_arnoldi_ritz(op, inner, b, m=120, nev=20)
    lam_s, Z_s, pair = K.select_deflation(op, op.gamma5, lam, Z)
    assert lam_s.size >= 4
    ev = np.linalg.eigvals(A)
    for l in lam_s:
        assert np.min(np.abs(ev - l)) < 1e-5
    # pairing is an involution; pairs are near-conjugate, singles near-real
    assert np.array_equal(pair[pair], np.arange(pair.size))
    for i, j in enumerate(pair):
        if i == j:
            assert abs(lam_s[i].imag) < K.IMAGLIM
        else:
            assert abs(lam_s[j] - np.conj(lam_s[i])) < K.IMAGLIM
        # u = gamma5 z_pair[i] is a left eigenvector of A for lam_i (dense check)
        u = op.gamma5(Z_s[:, j])
        assert np.linalg.norm(u.conj() @ A - lam_s[i] * u.conj()) < K.EVECTOL
        assert np.linalg.norm(A @ Z_s[:, i] - lam_s[i] * Z_s[:, i]) < K.EVECTOL


def test_left_right_projection(rng):
    # Sec. 2.1: the projected residual is orthogonal to U and x_hat + A^{-1} r = A^{-1} r0
    dims = (2, 2, 2, 2)
    op = operator(dims, "haar", 0, 0.12)
    A = dense(dims, "haar", 0, 0.12)
    Z = synth.random_block(op.n, 6, 1)
    U = synth.random_block(op.n, 6, 2)
    r0 = synth.random_block(op.n, 1, 3)[:, 0]
    xh, r, d = K.left_right_projection(op, Z, U, r0)
    assert np.linalg.norm(U.conj().T @ r) < 1e-11 * np.linalg.norm(r0)
    assert np.linalg.norm(xh + np.linalg.solve(A, r) - np.linalg.solve(A, r0)) < 1e-10 * np.linalg.norm(r0)
