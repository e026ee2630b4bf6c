"""Pins of the oracle's level samples, deflation, statistics and cost model."""

import json
import os

import numpy as np
import pytest

from conftest import dense, operator
from oracle import krylov as K
from oracle import mpmc as M
from oracle import philox
from oracle import polynomial as P
from paper_2306_09559_gb300 import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_deflation_identity_any_vectors(rng):
    # Tr(M - sum c z u^H) + sum c u^H z = Tr M, for any Z, U, c (Sec. 4.1)
    n, k = 60, 7
    Mx = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Z = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    U = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    c = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    defl_M = Mx - (Z * c) @ U.conj().T
    assert abs(np.trace(defl_M) + np.sum(c * np.einsum('ni,ni->i', U.conj(), Z)) - np.trace(Mx)) < 1e-10


def _small_setup(dims=(2, 2, 2, 4), kappa=0.14, seed=1):
    op = operator(dims, "haar", seed, kappa)
    A = dense(dims, "haar", seed, kappa)
    b0 = synth.random_unit_vector(op.n, 6)
    p_hi, p_lo, p_in = K.gmres_polynomials(op, b0, [14, 6, 3])
    p_out, _, _ = K.pp_gmres_roots(op, p_in, b0, m_out=4)
    lam, Z = K.pp_arnoldi_ritz(op, p_in, b0, m=120, nev=12)
    lam, Z, pair = K.select_deflation(op, op.gamma5, lam, Z)
    defl = M.Deflation(op, Z, lam, pair)
    polys = [{"kind": "composite", "inner": p_in, "outer": p_out},
             {"kind": "single", "roots": p_hi},
             {"kind": "single", "roots": p_lo}]
    return op, A, polys, defl


def _dense_of(A, spec, defl=None):
    op = lambda X: A @ X
    return M.apply_spec(op, spec, np.eye(A.shape[0], dtype=complex), defl)


def test_level_sample_matches_dense_formula():
    op, A, polys, defl = _small_setup()
    for level in range(3):
        s = M.level_samples(op, polys, level, seed=99, nsamples=3, defl=defl)
        Mhi = _dense_of(A, polys[level])
        Mlo = _dense_of(A, polys[level + 1]) if level + 1 < 3 else 0 * Mhi
        Md = Mhi - Mlo
        if level < 2:
            c = M.level_coefficients(polys, level, defl)
            Md = Md - (defl.Z * c) @ defl.U.conj().T
        for j in range(3):
            b = philox.z4_noise(99, level, j, op.n // 12)
            assert abs(s[j] - b.conj() @ Md @ b) < 1e-10 * op.n


def test_deflated_levels_unbiased_and_vs_dense_trace():
    # mean + exact correction estimates Tr(q_l - q_{l+1}) within 4 SE
    op, A, polys, defl = _small_setup()
    lam_A = np.linalg.eigvals(A)
    exact = [np.sum(M.spec_value(p, lam_A)) for p in polys]
    res = M.trace_levels(op, polys, seed=3, nsamples=400, defl=defl)
    for level in range(3):
        ex = exact[level] - (exact[level + 1] if level + 1 < 3 else 0)
        st = res[level]
        se_c = np.sqrt(st["var_complex"] / st["n"])
        assert abs(st["estimate"] - ex) < 4 * se_c + 1e-9 * op.n
    # deflation lowers the variance of the first difference level
    plain = M.statistics(M.level_samples(op, polys, 0, 3, 400, defl=None))
    assert res[0]["var_complex"] < plain["var_complex"]


def test_hutchinson_variance_closed_form():
    # Var(Re b^H M b) = 1/2 (sum_{i!=j} |M_ij|^2 + Re sum_{i!=j} M_ij M_ji) for Z4
    A = dense((2, 2, 2, 2), "haar", 0, 0.12)
    Minv = np.linalg.inv(A)
    N = 20000
    B = philox.z4_block(5, 0, 0, N, 16)
    s = np.einsum('nr,nm,mr->r', B.conj(), Minv, B)
    off = Minv - np.diag(np.diag(Minv))
    v_re = 0.5 * (np.sum(np.abs(off) ** 2) + np.real(np.sum(off * off.T)))
    v_c = np.sum(np.abs(off) ** 2)
    assert abs(s.mean() - np.trace(Minv)) < 4 * np.sqrt(v_c / N)
    assert abs(np.var(s.real, ddof=1) / v_re - 1) < 0.05
    assert abs(np.mean(np.abs(s - s.mean()) ** 2) / v_c - 1) < 0.05
    # diagonal of |b|^2 is exactly 1: a diagonal matrix has zero variance
    D = np.diag(np.diag(Minv))
    sd = np.einsum('nr,nm,mr->r', B.conj(), D, B)
    assert np.max(np.abs(sd - np.trace(D))) < 1e-12


def test_deflated_polynomial_maps_eigenvectors():
    # Sec. 4.3 read as M_1 = Z H^-1 U^H + p_1(A)(I - A Z H^-1 U^H): M_1 A Z = Z exactly
    op, A, polys, defl = _small_setup()
    spec = dict(polys[0], kind="deflated_composite")
    AZ = A @ defl.Z
    got = M.apply_spec(op, spec, AZ, defl)
    assert np.linalg.norm(got - defl.Z) < 1e-9 * np.linalg.norm(defl.Z)
    # and it is still a good approximate inverse: close to A^{-1} on a random vector
    v = synth.random_unit_vector(op.n, 77)
    x = M.apply_spec(op, spec, v, defl)
    assert np.linalg.norm(A @ x - v) < 0.2


def test_config1_two_level_estimate_vs_dense_lu():
    # 4^4 Haar links, kappa = 0.12: Tr(p_40) + Tr(A^{-1} - p_40) by Hutchinson
    dims, kappa = (4, 4, 4, 4), 0.12
    op = operator(dims, "haar", 0, kappa)
    A = dense(dims, "haar", 0, kappa)
    tr_exact = np.trace(np.linalg.inv(A))
    b0 = philox.z4_noise(0, 99, 0, 256) / np.sqrt(op.n)
    roots = K.gmres_polynomials(op, b0, [40])[0]
    N = 200
    B = philox.z4_block(1001, 0, 0, N, 256)
    pB = P.apply_poly(op, roots, B)
    s_poly = np.einsum('nr,nr->r', B.conj(), pB)
    B1 = philox.z4_block(1001, 1, 0, N, 256)
    s_rem = np.einsum('nr,nr->r', B1.conj(), np.linalg.solve(A, B1) - P.apply_poly(op, roots, B1))
    est = s_poly.mean() + s_rem.mean()
    se = np.sqrt(np.var(s_poly, ddof=1) / N + np.var(s_rem, ddof=1) / N)
    assert abs(est.real - tr_exact.real) < 4 * se
    # the remainder level carries far less variance than the polynomial level
    assert np.var(s_rem) < 0.05 * np.var(s_poly)


def test_multilevel_cost_table4():
    g = GOLDEN["table4_multilevel_cost"]
    eps = 0.0005 * 12 ** 3 * 16
    assert abs(eps - g["eps"]) < 1e-12
    h = M.hutchinson_cost(g["hutchinson"]["variance"], g["hutchinson"]["cost_per_noise"], eps)
    mp = M.multilevel_cost(g["multipoly"]["variances"], g["multipoly"]["costs_per_noise"], eps)
    # the table prints three significant digits
    assert abs(h / g["hutchinson"]["overall_cost"] - 1) < 0.005
    assert abs(mp / g["multipoly"]["overall_cost"] - 1) < 0.005


def test_per_noise_matvec_accounting_table4():
    g = GOLDEN["per_noise_matvecs"]
    mk = lambda d: {"kind": "single", "roots": np.ones(d + 1)}
    for d1, d2, cost in g["exact"]:
        assert M.spec_matvecs(mk(d1)) + M.spec_matvecs(mk(d2)) == cost
    for d1, d2, cost in g["within_one"]:
        # degree 359 = 30*12 - 1 composite (Table 2 caption)
        comp = {"kind": "deflated_composite", "inner": np.ones(30), "outer": np.ones(12)}
        assert abs(M.spec_matvecs(comp) + M.spec_matvecs(mk(d2)) - cost) <= 1


def test_statistics():
    """Values worked by hand: mean (6 + 2i)/4; real deviations -0.5, 0.5, 2.5, -2.5 (squares
    sum to 13, over n - 1 = 3); complex deviations with |.|^2 = 0.5, 2.5, 6.5, 8.5 (sum 18)."""
    s = np.array([1 + 1j, 2 - 1j, 4 + 0j, -1 + 2j])
    st = M.statistics(s)
    assert st["n"] == 4
    assert st["mean"] == 1.5 + 0.5j
    assert np.isclose(st["var_re"], 13.0 / 3.0, rtol=1e-15)
    assert np.isclose(st["var_complex"], 6.0, rtol=1e-15)
    assert np.isclose(st["se_re"], np.sqrt(13.0 / 12.0), rtol=1e-15)
    # a constant shift leaves the variances alone; a factor c scales the complex one by |c|^2
    sh = M.statistics(s + (3 - 7j))
    assert np.isclose(sh["var_re"], 13.0 / 3.0) and np.isclose(sh["var_complex"], 6.0)
    sc = M.statistics((2 - 1j) * s)
    assert np.isclose(sc["var_complex"], 5 * 6.0)
    # one sample: no variance
    one = M.statistics(np.array([2 + 1j]))
    assert one["mean"] == 2 + 1j and np.isnan(one["var_re"]) and np.isnan(one["se_re"])
