"""Seeded synthetic inputs: gauge fields and starting vectors.

This module holds none of the method's arithmetic.  It only draws the data
the method is run on, and it is the one module that both the CUDA path and
the CPU oracle consume.  The paper's workloads are quenched beta = 6.0
ensembles (Sec. 5, Examples 2 and 3) that are not available here; these
generators stand in for them:

* ``haar``: Haar-random SU(3) links (QR of a complex Gaussian matrix with
  the phase fix of Mezzadri, then division by a cube root of the
  determinant).
* ``near_identity``: U = proj_SU3(exp(i * eps * H)) with
  H = sum_a h_a lambda_a / 2 over the eight Gell-Mann matrices and
  h_a ~ N(0, 1); the exponential by Hermitian eigendecomposition, then
  one projection back onto SU(3) (polar factor, determinant fixed).
* ``unit``: all links equal to the identity (free field).

Random numbers come from numpy's PCG64 generator keyed by the seed, so the
fields are reproducible on any host.  Link arrays have shape
(4, Lt, Lz, Ly, Lx, 3, 3) complex128: U[mu, t, z, y, x, a, b].
"""

import numpy as np

_GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
_GELL_MANN[0][0, 1] = _GELL_MANN[0][1, 0] = 1
_GELL_MANN[1][0, 1], _GELL_MANN[1][1, 0] = -1j, 1j
_GELL_MANN[2][0, 0], _GELL_MANN[2][1, 1] = 1, -1
_GELL_MANN[3][0, 2] = _GELL_MANN[3][2, 0] = 1
_GELL_MANN[4][0, 2], _GELL_MANN[4][2, 0] = -1j, 1j
_GELL_MANN[5][1, 2] = _GELL_MANN[5][2, 1] = 1
_GELL_MANN[6][1, 2], _GELL_MANN[6][2, 1] = -1j, 1j
_GELL_MANN[7][0, 0] = _GELL_MANN[7][1, 1] = 1 / np.sqrt(3)
_GELL_MANN[7][2, 2] = -2 / np.sqrt(3)


def _fix_det(u):
    """Divide each 3x3 unitary by a cube root of its determinant."""
    det = np.linalg.det(u)
    return u / (det ** (1.0 / 3.0))[..., None, None]


def haar_su3(rng, count):
    """``count`` Haar-distributed SU(3) matrices."""
    z = (rng.standard_normal((count, 3, 3)) + 1j * rng.standard_normal((count, 3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    return _fix_det(q)


def near_identity_su3(rng, count, eps):
    """``count`` matrices proj_SU3(exp(i eps H)), H a Gaussian traceless Hermitian."""
    h = rng.standard_normal((count, 8))
    H = np.einsum('ka,aij->kij', h, _GELL_MANN) / 2
    w, v = np.linalg.eigh(H)
    u = np.einsum('kij,kj,klj->kil', v, np.exp(1j * eps * w), v.conj())
    # one projection back onto U(3) (polar factor), then onto SU(3)
    a, _, bh = np.linalg.svd(u)
    return _fix_det(a @ bh)


def gauge_field(dims, kind="haar", seed=0, eps=0.3):
    """Links for a lattice with dims = (Lx, Ly, Lz, Lt)."""
    lx, ly, lz, lt = dims
    count = 4 * lx * ly * lz * lt
    if kind == "unit":
        u = np.broadcast_to(np.eye(3, dtype=np.complex128), (count, 3, 3)).copy()
    else:
        rng = np.random.Generator(np.random.PCG64(seed))
        if kind == "haar":
            u = haar_su3(rng, count)
        elif kind == "near_identity":
            u = near_identity_su3(rng, count, eps)
        else:
            raise ValueError(f"unknown gauge field kind {kind!r}")
    return np.ascontiguousarray(u.reshape(4, lt, lz, ly, lx, 3, 3))


def random_unit_vector(n, seed):
    """Complex normal n-vector scaled to norm one (a Krylov starting vector)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return v / np.linalg.norm(v)


def random_block(n, nrhs, seed):
    """Complex normal n x nrhs block (generic right-hand sides for tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n, nrhs)) + 1j * rng.standard_normal((n, nrhs))


def gauge_transform(rng_seed, dims):
    """Random site-local SU(3) matrices g(x), shape (Lt, Lz, Ly, Lx, 3, 3)."""
    lx, ly, lz, lt = dims
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    return haar_su3(rng, lx * ly * lz * lt).reshape(lt, lz, ly, lx, 3, 3)
