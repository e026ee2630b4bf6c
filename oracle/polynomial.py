"""GMRES polynomials in root form (oracle; test infrastructure only).

A degree-d polynomial p with p(A) ~ A^{-1} comes from the GMRES residual
polynomial pi of degree m = d + 1 through pi(alpha) = 1 - alpha p(alpha)
(Sec. 3.1).  Its roots theta_1..theta_m are the harmonic Ritz values of the
GMRES run (see ``oracle/krylov.py``).  The paper applies p(A) to a vector
in the stable root form of its reference [PPGStable] (Sec. 2.3), which this
module reads as

    w_0 = v,   w_i = (I - A/theta_i) w_{i-1},
    p(A) v = sum_{i=1..m} theta_i^{-1} w_{i-1}          (m - 1 matvecs)

(the identity alpha * sum_i theta_i^{-1} w_{i-1}(alpha) = 1 - w_m(alpha)
= 1 - pi(alpha) makes this exactly p).  Roots are used in the order given;
``leja_order`` provides the modified Leja order that keeps high-degree
products stable.

The composite ("double") polynomial of Secs. 2.4 and 3.2 is
p_1(A) = p_in(A) p_out(A p_in(A)), of degree m_in * m_out - 1.
"""

import numpy as np


def leja_order(roots):
    """Modified Leja order of a root list (indices into ``roots``).

    First the root of largest modulus; then repeatedly the root that
    maximises the sum of log-distances to the roots already taken.  Ties go
    to the lowest original index.  Equal roots (distance 0) come last.
    """
    roots = np.asarray(roots, dtype=np.complex128)
    m = roots.size
    taken = np.zeros(m, dtype=bool)
    order = []
    first = int(np.argmax(np.abs(roots)))
    order.append(first)
    taken[first] = True
    score = np.zeros(m)
    for _ in range(1, m):
        last = roots[order[-1]]
        with np.errstate(divide='ignore'):
            score = score + np.log(np.abs(roots - last))
        cand = np.where(taken, -np.inf, score)
        # equal roots give -inf; fall back to the first untaken index
        if np.all(np.isneginf(cand[~taken])):
            nxt = int(np.flatnonzero(~taken)[0])
        else:
            nxt = int(np.argmax(cand))
        order.append(nxt)
        taken[nxt] = True
    return np.array(order, dtype=np.int64)


def apply_poly(op, roots, v):
    """p(A) v in root form; ``op`` applies A to a flat vector or block."""
    roots = np.asarray(roots, dtype=np.complex128)
    w = np.array(v, dtype=np.complex128)
    y = np.zeros_like(w)
    m = roots.size
    for i in range(m):
        y = y + w / roots[i]
        if i < m - 1:
            w = w - op(w) / roots[i]
    return y


def apply_residual_poly(op, roots, v):
    """pi(A) v = prod_i (I - A/theta_i) v  (m matvecs)."""
    w = np.array(v, dtype=np.complex128)
    for th in np.asarray(roots, dtype=np.complex128):
        w = w - op(w) / th
    return w


def residual_poly_coefficients(roots):
    """Power-basis coefficients c_0..c_m of pi(alpha) = prod (1 - alpha/theta_i)."""
    c = np.array([1.0 + 0j])
    for th in np.asarray(roots, dtype=np.complex128):
        # multiply by (1 - alpha/theta): new_k = c_k - c_{k-1}/theta
        nxt = np.zeros(c.size + 1, dtype=np.complex128)
        nxt[:-1] += c
        nxt[1:] -= c / th
        c = nxt
    return c


def poly_coefficients(roots):
    """Power-basis coefficients of p, from pi(alpha) = 1 - alpha p(alpha)."""
    c = residual_poly_coefficients(roots)
    return -c[1:]


def apply_poly_power_basis(op, coeffs, v):
    """sum_k coeffs[k] A^k v by Horner's rule (unstable at high degree)."""
    v = np.array(v, dtype=np.complex128)
    y = coeffs[-1] * v
    for ck in coeffs[-2::-1]:
        y = op(y) + ck * v
    return y


def poly_value(roots, lam):
    """p(lambda) in the same root form as :func:`apply_poly`, for scalars/arrays."""
    lam = np.asarray(lam, dtype=np.complex128)
    w = np.ones_like(lam)
    y = np.zeros_like(lam)
    roots = np.asarray(roots, dtype=np.complex128)
    for i, th in enumerate(roots):
        y = y + w / th
        if i < roots.size - 1:
            w = w * (1 - lam / th)
    return y


def residual_poly_value(roots, lam):
    """pi(lambda) = prod_i (1 - lambda/theta_i)."""
    lam = np.asarray(lam, dtype=np.complex128)
    out = np.ones_like(lam)
    for th in np.asarray(roots, dtype=np.complex128):
        out = out * (1 - lam / th)
    return out


def apply_composite(op, inner_roots, outer_roots, v):
    """p_in(A) p_out(A p_in(A)) v, materialising y = p_out(A p_in(A)) v first."""
    def B(w):
        return op(apply_poly(op, inner_roots, w))
    y = apply_poly(B, outer_roots, v)
    return apply_poly(op, inner_roots, y)


def composite_value(inner_roots, outer_roots, lam):
    """p_1(lambda) = p_in(lambda) p_out(lambda p_in(lambda))."""
    pin = poly_value(inner_roots, lam)
    return pin * poly_value(outer_roots, np.asarray(lam) * pin)


def composite_degree(m_in, m_out):
    """Degree of the double polynomial, (dp_in + 1)(dp_out + 1) - 1 (Sec. 3.2)."""
    return m_in * m_out - 1


def matvecs_single(m):
    """Products with A needed by :func:`apply_poly` with m roots."""
    return max(m - 1, 0)


def matvecs_composite(m_in, m_out):
    """Products with A needed by :func:`apply_composite`."""
    return (m_out - 1) * m_in + (m_in - 1)
