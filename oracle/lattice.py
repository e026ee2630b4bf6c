"""Wilson-Dirac matrix of a quenched lattice (oracle; test infrastructure only).

The paper works with "the quenched Wilson-Dirac fermion matrix" of size
n = 12 * volume (Sec. 5, Examples 2 and 3) and never writes it out.  This
module fixes the reading used throughout the project:

    (A psi)(x) = psi(x) - kappa * (H psi)(x)
    (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x)        psi(x + mu)
                        + (1 + gamma_mu) U_mu(x - mu)^+ psi(x - mu) ]

with Wilson parameter r = 1, so that kappa_c ~ 0.157 at beta = 6 as in
Example 2.  Gamma matrices are Hermitian, in the chiral DeGrand-Rossi
basis, with gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1).
Directions mu = 0, 1, 2, 3 are x, y, z, t.  The lattice is periodic in
all four directions; ``bc_t = -1`` makes it antiperiodic in t.

Storage (shared convention with the GPU library, each side implements it):
  * a vector is an array of shape (Lt, Lz, Ly, Lx, 4, 3) complex, optionally
    with a trailing right-hand-side axis; flattening it in C order gives the
    unknown index ((((t*Lz + z)*Ly + y)*Lx + x)*4 + spin)*3 + colour;
  * links are an array of shape (4, Lt, Lz, Ly, Lx, 3, 3): U[mu, site, a, b].

Everything is full 4x4 spin algebra with numpy einsum (no half-spinor
projection), so it shares no arithmetic with the GPU stencil.
"""

import numpy as np

_I = 1j

#: Hermitian gamma matrices gamma_1..gamma_4 (index 0..3), DeGrand-Rossi basis.
GAMMA = np.array([
    [[0, 0, 0, _I], [0, 0, _I, 0], [0, -_I, 0, 0], [-_I, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, _I, 0], [0, 0, 0, -_I], [-_I, 0, 0, 0], [0, _I, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)

#: gamma5 = gamma1 gamma2 gamma3 gamma4 (diag(1, 1, -1, -1) in this basis).
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]

_EYE4 = np.eye(4, dtype=np.complex128)

# numpy axis of each direction in a (Lt, Lz, Ly, Lx, ...) array
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def volume(dims):
    """Number of sites of a lattice with dims = (Lx, Ly, Lz, Lt)."""
    lx, ly, lz, lt = dims
    return lx * ly * lz * lt


def vector_shape(dims, nrhs=None):
    """Array shape of a spinor field (optionally a block of nrhs of them)."""
    lx, ly, lz, lt = dims
    base = (lt, lz, ly, lx, 4, 3)
    return base if nrhs is None else base + (nrhs,)


def _shift(psi, mu, sign, bc_t):
    """psi(x + sign*mu) on the periodic (or t-antiperiodic) torus."""
    ax = _AXIS[mu]
    out = np.roll(psi, -sign, axis=ax)
    if mu == 3 and bc_t != 1:
        # sites whose neighbour wrapped around the t boundary pick up bc_t
        sl = [slice(None)] * out.ndim
        sl[ax] = -1 if sign > 0 else 0
        out[tuple(sl)] *= bc_t
    return out


def apply_H(U, psi, bc_t=1):
    """Wilson hopping term H psi (the sum over mu above), full spinor algebra."""
    multi = psi.ndim == 7
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = _shift(psi, mu, +1, bc_t)
        bwd = _shift(psi, mu, -1, bc_t)
        U_here = U[mu]
        U_back = np.roll(U[mu], 1, axis=_AXIS[mu])  # U_mu(x - mu)
        if multi:
            col_f = np.einsum('tzyxab,tzyxsbr->tzyxsar', U_here, fwd)
            col_b = np.einsum('tzyxba,tzyxsbr->tzyxsar', U_back.conj(), bwd)
            out += np.einsum('pq,tzyxqar->tzyxpar', _EYE4 - GAMMA[mu], col_f)
            out += np.einsum('pq,tzyxqar->tzyxpar', _EYE4 + GAMMA[mu], col_b)
        else:
            col_f = np.einsum('tzyxab,tzyxsb->tzyxsa', U_here, fwd)
            col_b = np.einsum('tzyxba,tzyxsb->tzyxsa', U_back.conj(), bwd)
            out += np.einsum('pq,tzyxqa->tzyxpa', _EYE4 - GAMMA[mu], col_f)
            out += np.einsum('pq,tzyxqa->tzyxpa', _EYE4 + GAMMA[mu], col_b)
    return out


def apply_A(U, psi, kappa, bc_t=1):
    """A psi = psi - kappa H psi."""
    return psi - kappa * apply_H(U, psi, bc_t)


def apply_gamma5(psi):
    """gamma5 psi (acts on the spin index, axis -2 or -3 with rhs)."""
    if psi.ndim == 7:
        return np.einsum('pq,tzyxqar->tzyxpar', GAMMA5, psi)
    return np.einsum('pq,tzyxqa->tzyxpa', GAMMA5, psi)


def dense_A(U, kappa, bc_t=1, chunk=1024):
    """The n x n matrix A, column by column (tiny lattices only)."""
    lt, lz, ly, lx = U.shape[1:5]
    dims = (lx, ly, lz, lt)
    n = 12 * volume(dims)
    A = np.empty((n, n), dtype=np.complex128)
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        e = np.zeros((n, c1 - c0), dtype=np.complex128)
        e[np.arange(c0, c1), np.arange(c1 - c0)] = 1.0
        cols = apply_A(U, e.reshape(vector_shape(dims, c1 - c0)), kappa, bc_t)
        A[:, c0:c1] = cols.reshape(n, c1 - c0)
    return A


def flat(psi):
    """Vector (or block) as an n-vector (or n x nrhs matrix) in unknown order."""
    if psi.ndim == 7:
        return psi.reshape(-1, psi.shape[-1])
    return psi.reshape(-1)


def unflat(v, dims):
    """Inverse of :func:`flat`."""
    if v.ndim == 2:
        return v.reshape(vector_shape(dims, v.shape[1]))
    return v.reshape(vector_shape(dims))


class WilsonOperator:
    """A = I - kappa H as a callable on flat n-vectors or n x nrhs blocks."""

    def __init__(self, U, kappa, bc_t=1):
        self.U = np.asarray(U, dtype=np.complex128)
        self.kappa = float(kappa)
        self.bc_t = int(bc_t)
        lt, lz, ly, lx = self.U.shape[1:5]
        self.dims = (lx, ly, lz, lt)
        self.n = 12 * volume(self.dims)
        self.matvecs = 0  # number of single-vector products, as in the MVP columns

    def __call__(self, v):
        v = np.asarray(v, dtype=np.complex128)
        self.matvecs += 1 if v.ndim == 1 else v.shape[1]
        return flat(apply_A(self.U, unflat(v, self.dims), self.kappa, self.bc_t))

    def gamma5(self, v):
        return flat(apply_gamma5(unflat(np.asarray(v, dtype=np.complex128), self.dims)))
