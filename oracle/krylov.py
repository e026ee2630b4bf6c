"""Arnoldi / GMRES, harmonic Ritz roots and deflation eigenpairs (oracle).

Test infrastructure only.  Sources in the paper:

* GMRES residual polynomial pi(alpha) = 1 - alpha p(alpha); a degree-d p
  comes from stopping GMRES at iteration d + 1 (Sec. 3.1).  Its roots are
  the harmonic Ritz values of that GMRES run (Sec. 2.3, via [PPGStable]).
* The three single polynomials are read off one GMRES(maxit) cycle from a
  random normal unit vector at the proper iterations (Sec. 5, step 2a).
* p_out comes from PP(dp_in + 1)-GMRES, i.e. GMRES on A p_in(A) (Secs. 2.4,
  3.2); the deflated variant first applies one Left-right Projection to a
  Z4 starting vector (Secs. 2.1, 4.3; Sec. 5, step 2c).
* Eigenpairs come from PP-Arnoldi (regular Ritz pairs of A p_in(A)); left
  eigenvectors from gamma5 (Sec. 4); acceptance by the algorithm
  "Determine Eigenvalues and Eigenvectors for Deflation" (Sec. 4), with
  imaglim = 2e-4 and evectol = 1e-3.

Harmonic Ritz values at step m solve the generalized problem
(Hbar_m^H Hbar_m) y = theta H_m^H y, where Hbar_m is the (m+1) x m
Hessenberg matrix and H_m its leading m x m block (textbook definition; the
paper cites it).  This is evaluated with scipy.linalg.eig.
"""

import numpy as np
import scipy.linalg as sla

from . import polynomial as P

IMAGLIM = 2e-4   # Sec. 4: imaginary-part limit for "real" Ritz values
EVECTOL = 1e-3   # Sec. 4: residual limit for right and left Ritz vectors


def arnoldi(op, v0, m):
    """m steps of Arnoldi with modified Gram-Schmidt and one reorthogonalisation.

    Returns (V, Hbar, beta): V is n x (k+1), Hbar is (k+1) x k with k <= m
    (k < m only on breakdown), beta = ||v0||.
    """
    v0 = np.asarray(v0, dtype=np.complex128)
    n = v0.size
    beta = np.linalg.norm(v0)
    V = np.zeros((n, m + 1), dtype=np.complex128)
    H = np.zeros((m + 1, m), dtype=np.complex128)
    V[:, 0] = v0 / beta
    for j in range(m):
        w = op(V[:, j])
        for _ in range(2):          # MGS, then the same again (reorthogonalisation)
            for i in range(j + 1):
                h = np.vdot(V[:, i], w)
                H[i, j] += h
                w = w - h * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] == 0:
            return V[:, :j + 1], H[:j + 1, :j], beta
        V[:, j + 1] = w / H[j + 1, j]
    return V, H, beta


def gmres_least_squares(Hbar, beta):
    """y minimising ||beta e1 - Hbar y|| and the residual norm it leaves."""
    rhs = np.zeros(Hbar.shape[0], dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(Hbar, rhs, rcond=None)[0]
    return y, np.linalg.norm(rhs - Hbar @ y)


def gmres_iterate(V, Hbar, beta, m):
    """The GMRES solution x_m (x_0 = 0) after m steps, and its residual norm."""
    y, res = gmres_least_squares(Hbar[:m + 1, :m], beta)
    return V[:, :m] @ y, res


def harmonic_ritz(Hbar, m):
    """Harmonic Ritz values at step m from the leading (m+1) x m Hessenberg block."""
    Hb = Hbar[:m + 1, :m]
    Hm = Hb[:m, :m]
    vals = sla.eig(Hb.conj().T @ Hb, Hm.conj().T, right=False)
    return np.asarray(vals, dtype=np.complex128)


def gmres_polynomials(op, v0, degrees):
    """Roots (harmonic Ritz values) of the polynomials of the given degrees.

    One Arnoldi run to maxit = max(d) + 1 steps; the degree-d polynomial
    takes the d + 1 harmonic Ritz values at step d + 1.  Roots are returned
    in Leja order.
    """
    maxit = max(degrees) + 1
    V, Hbar, beta = arnoldi(op, v0, maxit)
    out = []
    for d in degrees:
        th = harmonic_ritz(Hbar, d + 1)
        out.append(th[P.leja_order(th)])
    return out


def gmres_residual_history(Hbar, beta):
    """Relative GMRES residual norm after each step 1..k."""
    k = Hbar.shape[1]
    return np.array([gmres_least_squares(Hbar[:j + 2, :j + 1], beta)[1] / beta
                     for j in range(k)])


def pp_operator(op, inner_roots):
    """v -> A p_in(A) v, the polynomial preconditioned operator."""
    return lambda v: op(P.apply_poly(op, inner_roots, v))


def pp_gmres_roots(op, inner_roots, v0, m_out=None, rtol=None, max_m=300):
    """Roots of p_out from GMRES on A p_in(A).

    Either a fixed number of roots ``m_out`` (harmonic Ritz values at step
    m_out) or, with ``rtol``, the first step whose relative residual is below
    rtol.  Returns (roots in Leja order, m_out, relative residual).
    """
    B = pp_operator(op, inner_roots)
    m = m_out if m_out is not None else max_m
    V, Hbar, beta = arnoldi(B, v0, m)
    if m_out is None:
        hist = gmres_residual_history(Hbar, beta)
        below = np.flatnonzero(hist < rtol)
        m_out = int(below[0]) + 1 if below.size else Hbar.shape[1]
    rel = gmres_least_squares(Hbar[:m_out + 1, :m_out], beta)[1] / beta
    th = harmonic_ritz(Hbar, m_out)
    return th[P.leja_order(th)], m_out, rel


def pp_arnoldi_ritz(op, inner_roots, v0, m, nev):
    """PP-Arnoldi: regular Ritz pairs of A p_in(A) nearest the origin.

    Returns (lam, Z): the nev Ritz vectors with the smallest Ritz values of
    A p_in(A), normalised, and for each the Rayleigh quotient
    lam_i = z_i^H A z_i as the eigenvalue estimate for A.
    """
    B = pp_operator(op, inner_roots)
    V, Hbar, _ = arnoldi(B, v0, m)
    k = Hbar.shape[1]
    mu, Y = np.linalg.eig(Hbar[:k, :k])
    idx = np.argsort(np.abs(mu), kind='stable')[:nev]
    Z = V[:, :k] @ Y[:, idx]
    Z = Z / np.linalg.norm(Z, axis=0)
    AZ = op(Z)
    lam = np.einsum('ni,ni->i', Z.conj(), AZ)
    return lam, Z


def select_deflation(op, gamma5, lam, Z, imaglim=IMAGLIM, evectol=EVECTOL):
    """The eigen-selection algorithm of Sec. 4.

    Candidates are visited in order of |lam|.  A value with |Im| < imaglim
    is real: accepted if the right residual ||A z - lam z|| and the left
    residual ||A^H u - conj(lam) u|| of u = gamma5 z are both below evectol.
    Otherwise it is accepted together with the next candidate if that is
    within imaglim of its conjugate and all four residuals (u_i = gamma5
    z_{i+1}, u_{i+1} = gamma5 z_i) are below evectol.

    Returns (lam_sel, Z_sel, pair): pair[i] = j means u_i = gamma5 z_j.
    """
    order = np.argsort(np.abs(lam), kind='stable')
    lam = lam[order]
    Z = Z[:, order]

    def right_res(i):
        z = Z[:, i]
        return np.linalg.norm(op(z) - lam[i] * z) / np.linalg.norm(z)

    def left_res(i, j):
        # u = gamma5 z_j as a left eigenvector for lam_i: A^H u = conj(lam_i) u,
        # and A^H = gamma5 A gamma5, so A^H u = gamma5 A z_j.
        u = gamma5(Z[:, j])
        ahu = gamma5(op(Z[:, j]))
        return np.linalg.norm(ahu - np.conj(lam[i]) * u) / np.linalg.norm(u)

    keep, pair = [], []
    i = 0
    while i < lam.size:
        if abs(lam[i].imag) < imaglim:
            if right_res(i) < evectol and left_res(i, i) < evectol:
                pair.append(len(keep))
                keep.append(i)
            i += 1
            continue
        if i + 1 < lam.size and abs(lam[i + 1] - np.conj(lam[i])) < imaglim:
            ok = (right_res(i) < evectol and right_res(i + 1) < evectol
                  and left_res(i, i + 1) < evectol and left_res(i + 1, i) < evectol)
            if ok:
                a = len(keep)
                keep += [i, i + 1]
                pair += [a + 1, a]
            i += 2
            continue
        i += 1
    keep = np.array(keep, dtype=np.int64)
    return lam[keep], Z[:, keep], np.array(pair, dtype=np.int64)


def left_right_projection(op, Z, U, r0):
    """Sec. 2.1: H = U^H A Z, c = U^H r0, H d = c; returns (x_hat, r, d)."""
    AZ = op(Z)
    H = U.conj().T @ AZ
    c = U.conj().T @ r0
    d = np.linalg.solve(H, c)
    return Z @ d, r0 - AZ @ d, d
