"""Deflated, polynomial-preconditioned GMRES (mpmc_solve) and the level
Tr(A^{-1} - p_1(A)) (mpmc_trace_inverse) against the oracle, which solves
with the dense matrix.  The solves stop at relative residual 1e-11; with the
condition number of these fields (< 100) the solutions agree to 1e-8
relative, and so do the samples (relative to their summed terms)."""

import numpy as np
import pytest

from conftest import dense
from oracle import mpmc as M
from oracle import philox
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G
from paper_2306_09559_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


@pytest.mark.parametrize("pin,defl", [(-1, False), (3, False), (3, True)])
def test_solve_matches_dense(pin, defl):
    from test_gpu_parity import handle, set_polys, small_setup
    op, polys, lam, Z, pair = small_setup()
    A = dense((4, 4, 4, 4), "haar", 0, 0.12)
    B = synth.random_block(op.n, 3, 21)
    with handle((4, 4, 4, 4)) as h:
        set_polys(h, polys)
        h.mpmc_set_poly(3, G.SINGLE, polys[0]["inner"], leja=False)
        if defl:
            h.mpmc_set_deflation(Z, lam, pair)
        X, rr, mv = h.mpmc_solve(B, pin=pin, rtol=1e-11, m=30, maxcycles=40)
    ref = np.linalg.solve(A, B)
    assert np.all(rr <= 1e-11)
    assert np.max(np.abs(X - ref)) <= 1e-8 * np.max(np.abs(ref))
    assert mv > 0


def test_trace_inverse_matches_oracle():
    from test_gpu_parity import handle, set_polys, small_setup
    op, polys, lam, Z, pair = small_setup()
    defl = M.Deflation(op, Z, lam, pair)
    A = dense((4, 4, 4, 4), "haar", 0, 0.12)
    N, first, seed = 7, 4, 55
    with handle((4, 4, 4, 4)) as h:
        set_polys(h, polys)
        h.mpmc_set_poly(3, G.SINGLE, polys[0]["inner"], leja=False)
        h.mpmc_set_deflation(Z, lam, pair)
        mean, var, s = h.mpmc_trace_inverse(1, seed, N, first, pin=3, rtol=1e-11, m=30, maxcycles=40)
    Bn = philox.z4_block(seed, 0xFFFF, first, N, op.n // 12)
    Xn = np.linalg.solve(A, Bn)
    p1 = polys[1]
    c = 1.0 / defl.lam - M.spec_value(p1, defl.lam)
    bx = np.einsum('nr,nr->r', Bn.conj(), Xn)
    bp = np.einsum('nr,nr->r', Bn.conj(), M.apply_spec(op, p1, Bn))
    dt = np.einsum('i,ir,ir->r', c, (defl.Z.conj().T @ Bn).conj(), defl.U.conj().T @ Bn)
    ref = bx - bp - dt
    scale = np.abs(bx) + np.abs(bp) + np.abs(dt)
    assert np.max(np.abs(s - ref) / scale) < 1e-8
    corr = np.sum(c * np.einsum('ni,ni->i', defl.U.conj(), defl.Z))
    assert abs(mean - (ref.mean() + corr)) < 1e-8 * np.max(scale)


def test_solve_rejects_reduced_precision():
    from test_gpu_parity import handle
    with handle((4, 4, 2, 4), prec=G.FP32) as h:
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_solve(np.ones(12 * 128, dtype=np.complex128))
        assert e.value.code == G.MPMC_ENOTSUP


def test_solve_without_cycles_reports_its_residual():
    """maxcycles = 0: only the Left-right Projection acts, x = Z H^{-1} U^H b.  It is an
    oblique projection (the residual norm may grow), and what it guarantees is the
    Petrov-Galerkin condition U^H (b - A x) = 0; the reported relative residual is that
    of the returned x."""
    from test_gpu_parity import handle, small_setup
    op, polys, lam, Z, pair = small_setup()
    defl = M.Deflation(op, Z, lam, pair)
    A = dense((4, 4, 4, 4), "haar", 0, 0.12)
    b = synth.random_block(op.n, 1, 5)[:, 0]
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        x, rr, mv = h.mpmc_solve(b, rtol=1e-12, m=10, maxcycles=0)
    r = b - A @ x
    res = np.linalg.norm(r) / np.linalg.norm(b)
    assert abs(rr[0] - res) < 1e-10
    assert np.max(np.abs(defl.U.conj().T @ r)) < 1e-10 * np.linalg.norm(b) * np.max(np.abs(defl.U))
