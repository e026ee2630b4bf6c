"""The whole multipolynomial estimate of Tr A^{-1} (Sec. 5, step 3 (a)-(e);
Eq. (2)) through the library: Tr(A^{-1} - M_1) by deflated PP-GMRES solves,
the two deflated difference levels with the sequential tolerance split, and
Tr(p_3) by probing with a distance-4 colouring.

The oracle replays the run on its own: the same noise vectors, its own
samples (dense solves, materialised polynomials), its own stopping rule
(tolerance eps/sqrt(3), then sqrt((eps^2 - currerr^2)/2), then
sqrt(eps^2 - currerr^2); check points 2, 3, ...; 3, 6, ...; 6, 9, ...) and its
own probing.  The stopping points must agree, the total must agree to 1e-10
of the summed level magnitudes, and it must lie within four reported
standard errors of Tr A^{-1} from a dense LU factorisation."""

import math

import numpy as np
import pytest
import scipy.linalg as sla

from conftest import dense, links, operator
from oracle import krylov as K
from oracle import mpmc as M
from oracle import philox
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import estimate as E
from paper_2306_09559_gb300 import mpmc as G
from paper_2306_09559_gb300 import synth

pytestmark = pytest.mark.gpu

DIMS, KAPPA, SEED = (4, 4, 4, 4), 0.12, 2024


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def _setup():
    op = operator(DIMS, "haar", 0, KAPPA)
    b0 = synth.random_unit_vector(op.n, 17)
    p2, p3, p_in = K.gmres_polynomials(op, b0, [20, 4, 6])
    p_out, _, _ = K.pp_gmres_roots(op, p_in, b0, m_out=8)
    lam, Z = K.pp_arnoldi_ritz(op, p_in, b0, m=120, nev=24)
    lam_s, Z_s, pair = K.select_deflation(op, op.gamma5, lam, Z)
    polys = [{"kind": "deflated_composite", "inner": p_in, "outer": p_out},
             {"kind": "single", "roots": p2}, {"kind": "single", "roots": p3}]
    return op, polys, p_in, lam_s, Z_s, pair


def _oracle_stop(re, tol, start, step):
    n = start
    while n <= len(re):
        if math.sqrt(np.var(re[:n], ddof=1) / n) <= tol:
            return n
        n += step
    raise AssertionError("the oracle replay needs more noise vectors")


@pytest.mark.parametrize("prec", [G.FP64, G.FP32])
def test_full_estimate_matches_the_oracle_and_dense_lu(prec):
    from test_gpu_parity import set_polys
    op, polys, p_in, lam, Z, pair = _setup()
    if prec != G.FP64:
        from conftest import fp32_polys
        polys = fp32_polys(polys)       # the polynomials an FP32 chain applies, on every side
    defl = M.Deflation(op, Z, lam, pair)
    A = dense(DIMS, "haar", 0, KAPPA)
    lu = sla.lu_factor(A)
    exact = np.trace(sla.lu_solve(lu, np.eye(A.shape[0], dtype=np.complex128)))
    V = op.n // 12
    # oracle samples of every Monte Carlo, far enough ahead for any stopping point
    NMAX = 96
    Bi = philox.z4_block(SEED, 0xFFFF, 0, NMAX, V)
    s_inv = (np.einsum('nr,nr->r', Bi.conj(), sla.lu_solve(lu, Bi))
             - np.einsum('nr,nr->r', Bi.conj(), M.apply_spec(op, polys[0], Bi, defl)))
    lev = [M.level_sample_parts(op, polys, l, SEED, NMAX, defl)[0] for l in (0, 1)]
    corr = [M.exact_correction(polys, l, defl) for l in (0, 1)]
    colours, nc = G.mpmc_colouring(DIMS, 4)
    probe = M.probing_trace_colours(op, polys[2], colours, nc)
    # a tolerance at which the Monte Carlo of largest variance needs about two dozen noise vectors
    # (each tolerance is about eps / sqrt(3)); every stopping point stays well inside NMAX
    var_max = max(np.var(x.real, ddof=1) for x in (s_inv, lev[0], lev[1]))
    eps = math.sqrt(3 * var_max / 24)
    # the oracle's own sequential replay (Sec. 5, step 3)
    n_o, est_o, err2 = [], [], 0.0
    for k, (s, c, start, step) in enumerate([(s_inv, 0.0, 2, 1), (lev[0], corr[0], 3, 3), (lev[1], corr[1], 6, 3)]):
        tol = math.sqrt(max(eps * eps - err2, 0.0) / (3 - k))
        n = _oracle_stop(s.real, tol, start, step)
        n_o.append(n)
        est_o.append(np.mean(s[:n]) + c)
        err2 += np.var(s[:n].real, ddof=1) / n
    total_o = sum(est_o) + probe

    with G.Handle(links(DIMS, "haar", 0, 0.3), KAPPA, G.FP64, 1) as h64, \
            G.Handle(links(DIMS, "haar", 0, 0.3), KAPPA, prec, 1) as hl:
        for h in (h64, hl):
            h.mpmc_set_deflation(Z, lam, pair)
            set_polys(h, polys)
        h64.mpmc_set_poly(3, G.SINGLE, p_in, leja=False)
        res = E.full_estimate(h64, hl, eps, SEED, pin=3, colours=colours, ncolours=nc, chunk=8, rtol=1e-12,
                              nmax=NMAX)
    n_g = [lv["n"] for lv in res["levels"]]
    assert res["err"] <= eps * (1 + 1e-12)
    scale = abs(probe) + sum(abs(x) for x in est_o)
    if prec == G.FP64:
        assert n_g == n_o
        assert abs(res["total"] - total_o) <= 1e-10 * scale, (res["total"], total_o)
        assert abs(res["probing"] - probe) <= 1e-11 * abs(probe)
    else:
        assert abs(res["levels"][0]["estimate"] - est_o[0]) <= 1e-8 * scale   # FP64 solves in both
        assert abs(res["probing"] - probe) <= 3e-6 * abs(probe)
    assert abs(res["total"].real - exact.real) <= 4 * res["err"], (res["total"], exact, res["err"])
