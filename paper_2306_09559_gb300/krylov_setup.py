"""Setup of the polynomials and deflation eigenpairs (Sec. 5, step 2).

All vector work (Arnoldi with two-pass classical Gram-Schmidt, products
with A and with p_in(A), Ritz-vector formation) runs in the library's FP64
CUDA kernels through the C ABI.  Only the small dense problems stay on the
host: eigenvalues of (m+1) x m Hessenberg matrices and the acceptance test
of the eigen-selection algorithm (Sec. 4).

* Harmonic Ritz values at GMRES step m are the eigenvalues of
  H_m + |h_{m+1,m}|^2 f e_m^T with f = H_m^{-H} e_m (the roots of the GMRES
  residual polynomial; Sec. 3.1 takes the degree-d polynomial from step
  d + 1).
* p_out: harmonic Ritz values of GMRES on A p_in(A) (Secs. 2.4, 3.2).
* Eigenpairs: regular Ritz pairs of A p_in(A) nearest the origin from
  PP-Arnoldi, eigenvalue estimate lambda = z^H A z for A, left vector
  gamma5 z (real lambda) or gamma5 of the conjugate partner; accepted when
  the right and left residual norms are below evectol, with |Im| < imaglim
  deciding "real" and pairing (Sec. 4; imaglim = 2e-4, evectol = 1e-3).
"""

import numpy as np

from . import mpmc as G

IMAGLIM = 2e-4
EVECTOL = 1e-3
# Smallest |d_i| = |z_pair(i)^H gamma5 z_i| (unit z) kept: the normalised left
# vector has norm 1/|d_i| and the deflation term of a sample grows with it.
DNORM_MIN = 1e-2


def harmonic_ritz(hbar, m):
    """Harmonic Ritz values at step m from the (m+1) x m Hessenberg block."""
    H = hbar[:m, :m]
    h = hbar[m, m - 1]
    em = np.zeros(m, dtype=np.complex128)
    em[-1] = 1.0
    f = np.linalg.solve(H.conj().T, em)
    return np.linalg.eigvals(H + (abs(h) ** 2) * np.outer(f, em))


def gmres_residual_norms(hbar):
    """Relative GMRES residual after each step (least squares on Hbar, beta = 1)."""
    k = hbar.shape[1]
    out = np.empty(k)
    for j in range(1, k + 1):
        Hb = hbar[:j + 1, :j]
        rhs = np.zeros(j + 1, dtype=np.complex128)
        rhs[0] = 1.0
        y = np.linalg.lstsq(Hb, rhs, rcond=None)[0]
        out[j - 1] = np.linalg.norm(rhs - Hb @ y)
    return out


class Setup:
    """Setup on an FP64 handle (its polynomial slots are used as scratch)."""

    SLOT = G.MAX_POLYS - 1

    def __init__(self, handle):
        if handle.precision != G.FP64:
            raise ValueError("setup needs an FP64 handle")
        self.h = handle

    def single_roots(self, v0, degrees):
        """Roots of the degree-d GMRES polynomials, one run to max(d) + 1 steps."""
        maxit = max(degrees) + 1
        hbar, steps = self.h.mpmc_arnoldi(-1, v0, maxit)
        if steps < maxit:
            raise RuntimeError(f"GMRES broke down after {steps} steps")
        return [harmonic_ritz(hbar, d + 1) for d in degrees]

    def pp_roots(self, inner_roots, v0, m_out=None, rtol=None, max_m=200):
        """Roots of p_out from GMRES on A p_in(A): fixed m_out, or the first step below rtol."""
        self.h.mpmc_set_poly(self.SLOT, G.SINGLE, inner_roots, leja=True)
        m = m_out if m_out is not None else max_m
        hbar, steps = self.h.mpmc_arnoldi(self.SLOT, v0, m)
        if m_out is None:
            res = gmres_residual_norms(hbar[:steps + 1, :steps])
            below = np.flatnonzero(res < rtol)
            m_out = int(below[0]) + 1 if below.size else steps
        return harmonic_ritz(hbar, m_out), m_out

    def ritz_pairs(self, inner_roots, v0, m, nev):
        """PP-Arnoldi Ritz vectors nearest the origin, kept on the device.

        Returns (lam, Zd, stats): Zd is a CUDA tensor (nev, n) of unit Ritz
        vectors of A p_in(A); stats[i] = (|z|^2, |Az|^2, Re z^H Az, Im z^H Az)
        from the library (A in FP64); lam_i = z_i^H A z_i / |z_i|^2.
        """
        import torch
        self.h.mpmc_set_poly(self.SLOT, G.SINGLE, inner_roots, leja=True)
        basis = torch.zeros((m + 1, self.h.n), dtype=torch.complex128, device="cuda")
        hbar, steps = self.h.mpmc_arnoldi(self.SLOT, v0, m, basis=basis)
        k = steps
        mu, Y = np.linalg.eig(hbar[:k, :k])
        idx = np.argsort(np.abs(mu), kind="stable")[:nev]
        Zd = torch.zeros((idx.size, self.h.n), dtype=torch.complex128, device="cuda")
        self.h.mpmc_combine(basis, k, Y[:, idx], Zd)
        torch.cuda.synchronize()
        del basis
        stats = self.h.mpmc_vector_stats(Zd)
        lam = (stats[:, 2] + 1j * stats[:, 3]) / stats[:, 0]
        return lam, Zd, stats

    @staticmethod
    def select(lam, stats, imaglim=IMAGLIM, evectol=EVECTOL, kmax=None):
        """The acceptance rule of Sec. 4 on candidates sorted by |lambda|.

        Residual norms come from the per-vector statistics in closed form:
        |A z - mu z|^2 = |Az|^2 - 2 Re(conj(mu) z^H A z) + |mu|^2 |z|^2.  The
        left residual of u = gamma5 z_j for eigenvalue lambda_i is
        |A^H u - conj(lambda_i) u| = |A z_j - conj(lambda_i) z_j| because
        A^H = gamma5 A gamma5 and gamma5 is unitary.
        Returns (indices into the candidates, pair map of the kept list).
        """
        zz, aa, zaz = stats[:, 0], stats[:, 1], stats[:, 2] + 1j * stats[:, 3]

        def res(i, val):
            r2 = aa[i] - 2 * np.real(np.conj(val) * zaz[i]) + abs(val) ** 2 * zz[i]
            return np.sqrt(max(r2, 0.0) / zz[i])

        order = np.argsort(np.abs(lam), kind="stable")
        keep, pair = [], []
        p = 0
        while p < order.size and (kmax is None or len(keep) < kmax):
            i = order[p]
            if abs(lam[i].imag) < imaglim:
                if res(i, lam[i]) < evectol and res(i, np.conj(lam[i])) < evectol:
                    pair.append(len(keep))
                    keep.append(i)
                p += 1
            elif p + 1 < order.size and abs(lam[order[p + 1]] - np.conj(lam[i])) < imaglim:
                j = order[p + 1]
                ok = (res(i, lam[i]) < evectol and res(j, lam[j]) < evectol
                      and res(j, np.conj(lam[i])) < evectol and res(i, np.conj(lam[j])) < evectol)
                if ok and (kmax is None or len(keep) + 2 <= kmax):
                    a = len(keep)
                    keep += [i, j]
                    pair += [a + 1, a]
                p += 2
            else:
                p += 1
        return np.array(keep, dtype=np.int64), np.array(pair, dtype=np.int32)

    def eigenpairs(self, inner_roots, v0, m, ndefinit, kmax=None, imaglim=IMAGLIM, evectol=EVECTOL):
        """(Zd, lam, pair): accepted eigenvectors as a CUDA tensor (k, n), eigenvalues, pairing."""
        import torch
        lam, Zd, stats = self.ritz_pairs(inner_roots, v0, m, ndefinit)
        keep, pair = self.select(lam, stats, imaglim, evectol, kmax)
        Zsel = Zd[torch.as_tensor(keep, device=Zd.device)].contiguous() if keep.size else Zd[:0]
        return Zsel, lam[keep], pair

    @staticmethod
    def well_conditioned(d, pair, dmin=DNORM_MIN):
        """Indices of the pairs to keep: |d_i| >= dmin for i and its partner.

        Returns (keep, new pair map of the kept list).
        """
        ok = np.abs(d) >= dmin
        ok &= ok[pair]                      # a conjugate pair stays or goes together
        keep = np.flatnonzero(ok)
        pos = -np.ones(len(d), dtype=np.int64)
        pos[keep] = np.arange(keep.size)
        return keep, pos[pair[keep]].astype(np.int32)

    def projected_start(self, seed):
        """A Z4 vector after one Left-right Projection, normalised (Sec. 5, step 2c).

        Needs the deflation vectors set on the setup handle.
        """
        b = self.h.mpmc_noise(seed, 99, 0, 1)
        r = self.h.mpmc_project(b)[:, 0]
        return r / np.linalg.norm(r)
