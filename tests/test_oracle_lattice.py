"""Pins of the oracle's Wilson-Dirac matrix against mathematics it does not contain."""

import itertools

import numpy as np
import pytest

from conftest import dense, links, operator
from oracle import lattice as L
from paper_2306_09559_gb300 import synth


def test_gamma_algebra():
    # Clifford algebra, hermiticity, and gamma5 diagonal (the basis convention)
    for a, b in itertools.product(range(4), repeat=2):
        ac = L.GAMMA[a] @ L.GAMMA[b] + L.GAMMA[b] @ L.GAMMA[a]
        assert np.allclose(ac, 2 * np.eye(4) * (a == b), atol=0)
    for g in L.GAMMA:
        assert np.array_equal(g, g.conj().T)
    assert np.array_equal(L.GAMMA5, np.diag([1, 1, -1, -1]).astype(complex))


@pytest.mark.parametrize("bc_t", [1, -1])
def test_gamma5_hermiticity_dense(bc_t):
    # gamma5 A gamma5 = A^H (Sec. 4 relies on it for the left eigenvectors)
    A = dense((2, 2, 2, 2), "haar", 0, 0.13, 0.3, bc_t)
    g5 = np.kron(np.eye(16), np.kron(np.diag([1, 1, -1, -1]), np.eye(3)))
    assert np.max(np.abs(g5 @ A @ g5 - A.conj().T)) < 1e-14


def _free_eigs(dims, kappa, bc_t=1):
    lx, ly, lz, lt = dims
    out = []
    for n in itertools.product(range(lx), range(ly), range(lz), range(lt)):
        p = [2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
             (2 * np.pi * n[3] + (np.pi if bc_t == -1 else 0)) / lt]
        a = 1 - 2 * kappa * sum(np.cos(p))
        b = 2 * kappa * np.sqrt(sum(np.sin(q) ** 2 for q in p))
        out += [a + 1j * b] * 6 + [a - 1j * b] * 6
    return np.array(out)


@pytest.mark.parametrize("dims,bc_t", [((2, 2, 2, 2), 1), ((3, 3, 2, 4), 1), ((2, 3, 2, 4), -1)])
def test_free_field_spectrum(dims, bc_t):
    # U = 1: eigenvalues 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p), each 6-fold
    kappa = 0.11
    A = L.dense_A(synth.gauge_field(dims, "unit"), kappa, bc_t)
    ev = np.sort_complex(np.round(np.linalg.eigvals(A), 10))
    ref = np.sort_complex(np.round(_free_eigs(dims, kappa, bc_t), 10))
    assert np.max(np.abs(ev - ref)) < 1e-9


def test_free_field_trace_inverse_4444():
    dims, kappa = (4, 4, 4, 4), 0.12
    A = L.dense_A(synth.gauge_field(dims, "unit"), kappa)
    tr = np.trace(np.linalg.inv(A))
    ref = np.sum(1.0 / _free_eigs(dims, kappa))
    assert abs(tr - ref) < 1e-9 * abs(ref)
    assert abs(ref.imag) < 1e-9


def test_traces_of_A_and_A_squared():
    # Tr H = 0 always; Tr H^2 = 0 for L >= 3 since (1+g)(1-g) = 0
    A = dense((3, 3, 3, 3), "haar", 1, 0.12)
    n = A.shape[0]
    assert abs(np.trace(A) - n) < 1e-12
    assert abs(np.sum(A * A.T) - n) < 1e-9


def test_trace_A_squared_fails_on_2444_by_design():
    # on a 2-site direction x+mu = x-mu, so back-and-forth hops no longer cancel
    A = dense((2, 2, 2, 2), "haar", 0, 0.12)
    assert abs(np.sum(A * A.T) - A.shape[0]) > 1e-3


def test_gauge_covariance():
    # A(U^g) = G A G^+ with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^+
    dims = (4, 4, 4, 4)
    U = links(dims, "haar", 2)
    g = synth.gauge_transform(7, dims)
    Ug = np.empty_like(U)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=axis[mu])
        Ug[mu] = np.einsum('tzyxab,tzyxbc,tzyxdc->tzyxad', g, U[mu], g_fwd.conj())
    psi = synth.random_block(12 * 256, 1, 3)[:, 0].reshape(L.vector_shape(dims))
    lhs = L.apply_A(Ug, np.einsum('tzyxab,tzyxsb->tzyxsa', g, psi), 0.12)
    rhs = np.einsum('tzyxab,tzyxsb->tzyxsa', g, L.apply_A(U, psi, 0.12))
    assert np.max(np.abs(lhs - rhs)) < 1e-13


def test_trace_inverse_real_and_gauge_invariant():
    A = dense((2, 2, 2, 2), "haar", 3, 0.14)
    tr = np.trace(np.linalg.inv(A))
    assert abs(tr.imag) < 1e-10 * abs(tr)


def test_block_apply_matches_columns():
    op = operator((4, 4, 2, 4), "haar", 0, 0.12)
    X = synth.random_block(op.n, 5, 11)
    Y = op(X)
    for j in range(5):
        assert np.max(np.abs(Y[:, j] - op(X[:, j]))) < 1e-13


def test_dense_matches_matvec_and_index_order():
    # column c of the dense matrix is A e_c with e_c in the documented unknown order
    dims = (2, 2, 2, 2)
    A = dense(dims, "haar", 0, 0.12)
    op = operator(dims, "haar", 0, 0.12)
    v = synth.random_block(op.n, 1, 5)[:, 0]
    assert np.max(np.abs(A @ v - op(v))) < 1e-13
    # the unknown ((((t*Lz+z)*Ly+y)*Lx+x)*4+s)*3+c couples only to its own site
    # and the 8 nearest neighbours
    lx, ly, lz, lt = dims
    x, y, z, t, s, c = 1, 0, 1, 0, 2, 1
    col = ((((t * lz + z) * ly + y) * lx + x) * 4 + s) * 3 + c
    sites = set(np.flatnonzero(np.abs(A[:, col]) > 0) // 12)
    nbrs = {((t * lz + z) * ly + y) * lx + x}
    for d in range(4):
        for sg in (1, -1):
            q = [x, y, z, t]
            q[d] = (q[d] + sg) % dims[d]
            nbrs.add(((q[3] * lz + q[2]) * ly + q[1]) * lx + q[0])
    assert sites == nbrs


def test_synthetic_links_are_su3():
    for kind in ("haar", "near_identity"):
        U = synth.gauge_field((2, 2, 2, 4), kind, seed=4, eps=0.3).reshape(-1, 3, 3)
        assert np.max(np.abs(U @ U.conj().transpose(0, 2, 1) - np.eye(3))) < 1e-13
        assert np.max(np.abs(np.linalg.det(U) - 1)) < 1e-13
    Un = synth.gauge_field((2, 2, 2, 4), "near_identity", seed=4, eps=0.05).reshape(-1, 3, 3)
    assert np.max(np.abs(Un - np.eye(3))) < 0.2
