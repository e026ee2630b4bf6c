"""Multipolynomial Monte Carlo level samples and statistics (oracle).

Test infrastructure only.  The method (Sec. 3.1, Eq. (2)):

    Tr A^{-1} = Tr(A^{-1} - p_1) + Tr(p_1 - p_2) + Tr(p_2 - p_3) + Tr(p_3)

Each trace on the right is a Hutchinson Monte Carlo over Z4 noise b with
samples b^H M b (Sec. 1; the b^T printed there is read as b^H, the form
used in Secs. 4.1 and 5).  The difference levels are deflated (Sec. 4.1):

    Tr(p_l - p_{l+1} - sum_i c_i z_i u_i^H) + sum_i c_i u_i^H z_i,
    c_i = p_l(lambda_i) - p_{l+1}(lambda_i),

with u_i the gamma5 left eigenvector of Sec. 4, scaled so u_i^H z_i = 1.
The subtracted part's trace is added back exactly.

Levels in this module follow the project's reading of the configurations:
with polynomials q_0, ..., q_{L-1} (highest degree first), level l < L-1 is
Tr(q_l - q_{l+1}) (deflated when eigenpairs are given) and level L-1 is
Tr(q_{L-1}) by plain Hutchinson.  Level l draws its noise with Philox
level id l, noise index j = 0, 1, ...

A polynomial is a dict:
  {"kind": "single", "roots": theta}
  {"kind": "composite", "inner": theta, "outer": eta}
  {"kind": "deflated_composite", "inner": theta, "outer": eta}
The deflated composite is Sec. 4.3 read as
M_1 = Z H^{-1} U^H + p_1(A) (I - A Z H^{-1} U^H), H = U^H A Z: a
Left-right Projection (Sec. 2.1) followed by the polynomial on the
projected residual.  It maps z_i to z_i / lambda_i, so its deflation
coefficient is c_i = 1/lambda_i - p_{l+1}(lambda_i).
"""

import numpy as np

from . import polynomial as P
from . import philox


class Deflation:
    """Right eigenvectors Z (n x k), eigenvalues lam, pairing u_i = gamma5 z_pair[i].

    The left vectors are scaled so that u_i^H z_i = 1 (Sec. 2.2 uses
    z_i u_i^* with that normalisation implied).
    """

    def __init__(self, op, Z, lam, pair):
        self.Z = np.asarray(Z, dtype=np.complex128)
        self.lam = np.asarray(lam, dtype=np.complex128)
        self.pair = np.asarray(pair, dtype=np.int64)
        g5Zp = op.gamma5(self.Z[:, self.pair])
        d = np.einsum('ni,ni->i', g5Zp.conj(), self.Z)      # (gamma5 z_pair)^H z
        self.U = g5Zp / np.conj(d)[None, :]
        self._op = op
        self._Hinv = None

    @property
    def k(self):
        return self.lam.size

    def projection(self):
        """H^{-1} with H = U^H A Z (k x k), formed on first use."""
        if self._Hinv is None:
            AZ = self._op(self.Z)
            self._AZ = AZ
            self._Hinv = np.linalg.inv(self.U.conj().T @ AZ)
        return self._Hinv, self._AZ


def apply_spec(op, spec, v, defl=None):
    """M v for a polynomial spec (flat n-vector or n x r block)."""
    kind = spec["kind"]
    if kind == "single":
        return P.apply_poly(op, spec["roots"], v)
    if kind == "composite":
        return P.apply_composite(op, spec["inner"], spec["outer"], v)
    if kind == "deflated_composite":
        Hinv, AZ = defl.projection()
        d = Hinv @ (defl.U.conj().T @ v)
        r = v - AZ @ d
        return defl.Z @ d + P.apply_composite(op, spec["inner"], spec["outer"], r)
    raise ValueError(kind)


def spec_value(spec, lam):
    """The scalar the level's deflation coefficient uses for eigenvalue lam."""
    kind = spec["kind"]
    if kind == "single":
        return P.poly_value(spec["roots"], lam)
    if kind == "composite":
        return P.composite_value(spec["inner"], spec["outer"], lam)
    if kind == "deflated_composite":
        return 1.0 / np.asarray(lam, dtype=np.complex128)
    raise ValueError(kind)


def spec_matvecs(spec):
    """Products with A per vector, the MVP count of Tables 1-8."""
    kind = spec["kind"]
    if kind == "single":
        return P.matvecs_single(len(spec["roots"]))
    return P.matvecs_composite(len(spec["inner"]), len(spec["outer"]))


def level_coefficients(polys, level, defl):
    """c_i of level ``level`` (zeros for the last, undeflated level)."""
    if defl is None or level == len(polys) - 1:
        return np.zeros(0 if defl is None else defl.k, dtype=np.complex128)
    return spec_value(polys[level], defl.lam) - spec_value(polys[level + 1], defl.lam)


def level_sample_terms(op, polys, level, b, defl=None):
    """The three pieces of one sample: (b^H q_l b, b^H q_{l+1} b, deflation term)."""
    hi = np.vdot(b, apply_spec(op, polys[level], b, defl))
    if level + 1 < len(polys):
        lo = np.vdot(b, apply_spec(op, polys[level + 1], b, defl))
    else:
        lo = 0.0 + 0j
    dterm = 0.0 + 0j
    if defl is not None and level + 1 < len(polys):
        c = level_coefficients(polys, level, defl)
        bz = defl.Z.conj().T @ b          # b^H z_i = conj(z_i^H b)
        ub = defl.U.conj().T @ b          # u_i^H b
        dterm = np.sum(c * np.conj(bz) * ub)
    return hi, lo, dterm


def level_samples(op, polys, level, seed, nsamples, defl=None, first=0, block=32):
    """Samples s_j = b_j^H (q_l - q_{l+1}) b_j - deflation term, j = first..first+N-1.

    Noise vectors are processed ``block`` at a time as the columns of an
    n x block matrix; every column is handled exactly as a single vector
    would be (the products with A act column by column).
    """
    return level_sample_parts(op, polys, level, seed, nsamples, defl, first, block)[0]


def level_sample_parts(op, polys, level, seed, nsamples, defl=None, first=0, block=32):
    """(samples, b^H q_l b, b^H q_{l+1} b, deflation terms) for noises first..first+N-1."""
    nsites = op.n // 12
    hi = np.empty(nsamples, dtype=np.complex128)
    lo = np.zeros(nsamples, dtype=np.complex128)
    dt = np.zeros(nsamples, dtype=np.complex128)
    for j0 in range(0, nsamples, block):
        cnt = min(block, nsamples - j0)
        B = philox.z4_block(seed, level, first + j0, cnt, nsites)
        hi[j0:j0 + cnt] = np.einsum('nr,nr->r', B.conj(), apply_spec(op, polys[level], B, defl))
        if level + 1 < len(polys):
            lo[j0:j0 + cnt] = np.einsum('nr,nr->r', B.conj(),
                                        apply_spec(op, polys[level + 1], B, defl))
            if defl is not None:
                c = level_coefficients(polys, level, defl)
                bz = (defl.Z.conj().T @ B).conj()      # b^H z_i
                ub = defl.U.conj().T @ B               # u_i^H b
                dt[j0:j0 + cnt] = np.einsum('i,ir,ir->r', c, bz, ub)
    return hi - lo - dt, hi, lo, dt


def exact_correction(polys, level, defl):
    """sum_i c_i u_i^H z_i, the deflated part's exact trace (= sum_i c_i)."""
    if defl is None or level == len(polys) - 1:
        return 0.0 + 0j
    c = level_coefficients(polys, level, defl)
    uz = np.einsum('ni,ni->i', defl.U.conj(), defl.Z)
    return np.sum(c * uz)


def statistics(samples):
    """Mean (complex), sample variance of the real parts, complex variance, SE of Re."""
    s = np.asarray(samples, dtype=np.complex128)
    n = s.size
    mean = s.mean()
    var_re = np.var(s.real, ddof=1) if n > 1 else np.nan
    var_c = np.sum(np.abs(s - mean) ** 2) / (n - 1) if n > 1 else np.nan
    return {"mean": mean, "var_re": var_re, "var_complex": var_c,
            "se_re": np.sqrt(var_re / n) if n > 1 else np.nan, "n": n}


def trace_levels(op, polys, seed, nsamples, defl=None):
    """Per-level estimate (mean + exact correction) and statistics."""
    out = []
    for level in range(len(polys)):
        s = level_samples(op, polys, level, seed, nsamples, defl)
        st = statistics(s)
        st["correction"] = exact_correction(polys, level, defl)
        st["estimate"] = st["mean"] + st["correction"]
        st["samples"] = s
        out.append(st)
    return out


def multilevel_cost(variances, costs, eps):
    """Eq. (3): C = eps^-2 (sum_l sqrt(V_l C_l))^2."""
    v = np.asarray(variances, dtype=np.float64)
    c = np.asarray(costs, dtype=np.float64)
    return float(np.sum(np.sqrt(v * c)) ** 2 / eps ** 2)


def hutchinson_cost(variance, cost, eps):
    """Plain Monte Carlo cost eps^-2 V_0 C_0 (Sec. 5, after Eq. (3))."""
    return float(variance * cost / eps ** 2)


def probing_vectors(dims, m, cols):
    """Probe vectors for the distance colouring of period m (m divides every extent).

    Column q = 12 * colour + e, colour = x%m + m (y%m) + m^2 (z%m) + m^3 (t%m):
    v_q(site, e') = 1 where the site has that colour and e' = e, else 0.
    Two sites of one colour differ by a multiple of m in every direction, so
    they are at least m hops apart on the periodic lattice.
    """
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    colour = ((x % m) + m * (y % m) + m * m * (z % m) + m ** 3 * (t % m)).reshape(-1)
    V = colour.size
    out = np.zeros((V, 12, len(cols)), dtype=np.complex128)
    for j, q in enumerate(cols):
        c, e = divmod(q, 12)
        out[colour == c, e, j] = 1.0
    return out.reshape(12 * V, len(cols))


def probing_trace(op, spec, m, defl=None, block=48):
    """Sum over the 12 m^4 probe vectors of v^H p(A) v: the probing estimate of
    Tr p(A) (exact when p(A) couples no two sites that are m or more hops apart,
    i.e. for polynomials of degree below m)."""
    dims = op.dims
    if any(L % m for L in dims):
        raise ValueError("m must divide every lattice extent")
    total = 0j
    nq = 12 * m ** 4
    for q0 in range(0, nq, block):
        cols = list(range(q0, min(nq, q0 + block)))
        Vb = probing_vectors(dims, m, cols)
        total += np.einsum('nr,nr->', Vb.conj(), apply_spec(op, spec, Vb, defl))
    return total


def torus_distance(dims, a, b):
    """Hop distance between sites a and b (site index x fastest) of the periodic
    lattice: the sum over directions of the shorter way round."""
    d = 0
    for L in dims:
        xa, xb = a % L, b % L
        a, b = a // L, b // L
        r = abs(xa - xb)
        d += min(r, L - r)
    return d


def distance_colouring(dims, distance):
    """A distance-`distance` colouring of the graph of A (Sec. 3.1, choice of
    p_3): sites whose hop distance on the periodic lattice is at most
    `distance` receive different colours.  Plain greedy colouring in site
    order, every earlier site checked by its hop distance (small lattices
    only).  Returns (colours as an int array of V entries, number of colours)."""
    V = int(np.prod(dims))
    colours = np.full(V, -1, dtype=np.int64)
    for s in range(V):
        taken = {colours[r] for r in range(s) if torus_distance(dims, s, r) <= distance}
        c = 0
        while c in taken:
            c += 1
        colours[s] = c
    return colours, int(colours.max()) + 1


def probing_vectors_colours(colours, cols):
    """Probe vectors of an arbitrary site colouring: column q = 12 c + e is the
    indicator of {sites of colour c} x {spin-colour component e}."""
    colours = np.asarray(colours)
    V = colours.size
    out = np.zeros((V, 12, len(cols)), dtype=np.complex128)
    for j, q in enumerate(cols):
        c, e = divmod(q, 12)
        out[colours == c, e, j] = 1.0
    return out.reshape(12 * V, len(cols))


def probing_trace_colours(op, spec, colours, ncolours, defl=None, block=48):
    """Sum over the 12 * ncolours probe vectors of v^H p(A) v.  Exact when no
    two sites of one colour are coupled by p(A), i.e. when same-coloured sites
    are more hops apart than the degree of p."""
    total = 0j
    nq = 12 * ncolours
    for q0 in range(0, nq, block):
        cols = list(range(q0, min(nq, q0 + block)))
        Vb = probing_vectors_colours(colours, cols)
        total += np.einsum('nr,nr->', Vb.conj(), apply_spec(op, spec, Vb, defl))
    return total
