"""Workloads (seeded synthetic lattices with their polynomial levels) and their setup.

Each workload names its lattice, gauge-field generator, kappa, the levels
(highest degree first, Eq. (2)), the number of deflation eigenpairs and the
noise vectors per level.  A composite level (m_in, m_out) has m_in roots
of p_in and m_out roots of p_out, degree m_in * m_out - 1 (Sec. 3.2).

``setup`` runs Sec. 5, step 2 with the library's FP64 GPU kernels
(:mod:`.krylov_setup`): one GMRES run for the single polynomials and p_in,
GMRES on A p_in(A) for p_out, PP-Arnoldi plus the Sec. 4 acceptance rule
for the eigenpairs.
"""

from dataclasses import dataclass, field

import numpy as np

from . import krylov_setup
from . import mpmc as G
from . import synth


@dataclass(frozen=True)
class Workload:
    key: str
    dims: tuple
    links: str
    gauge_seed: int
    eps: float
    kappa: float
    levels: tuple            # ("single", d) or ("composite", m_in, m_out)
    k: int                   # deflation eigenpairs
    nsamples: int            # Z4 noise vectors per level
    noise_seed: int
    setup_seed: int
    arnoldi_m: int = 0       # PP-Arnoldi steps for the eigenpairs
    ndefinit: int = 0        # Ritz values considered (Sec. 4)
    block: int = 64          # right-hand sides per launch

    @property
    def V(self):
        lx, ly, lz, lt = self.dims
        return lx * ly * lz * lt

    @property
    def n(self):
        return 12 * self.V

    def degrees(self):
        return [lv[1] if lv[0] == "single" else lv[1] * lv[2] - 1 for lv in self.levels]

    def applies_per_step(self):
        """Noise-vector polynomial applications in one pass over all levels."""
        L = len(self.levels)
        return self.nsamples * (2 * (L - 1) + 1)

    def matvecs_per_step(self):
        mv = []
        for lv in self.levels:
            mv.append(lv[1] if lv[0] == "single" else lv[1] * lv[2] - 1)
        L = len(mv)
        return self.nsamples * sum(mv[l] + (mv[l + 1] if l + 1 < L else 0) for l in range(L))

    def describe(self):
        lx, ly, lz, lt = self.dims
        lat = f"{lx}x{ly}x{lz}x{lt}"
        lv = []
        for x in self.levels:
            if x[0] == "single":
                lv.append(f"deg{x[1]}")
            else:
                tag = "projected-composite" if x[0] == "deflated_composite" else "composite"
                lv.append(f"{tag}{x[2]}x{x[1]}=deg{x[1] * x[2] - 1}")
        return (f"Wilson-Dirac {lat} {self.links} eps={self.eps} kappa={self.kappa}; levels "
                f"[{', '.join(lv)}]; {self.k} deflation eigenpairs; {self.nsamples} Z4 noises/level")


WORKLOADS = {
    # the small plain FP64 case: one degree-40 polynomial on a 4^4 Haar field
    "4^4": Workload("4^4", (4, 4, 4, 4), "haar", 0, 0.0, 0.12, (("single", 40),), 0, 200, 1001, 2001,
                    block=40),
    # the headline multipolynomial case: 8^4, three levels, 50 eigenpairs, 512 noises/level
    "8^4": Workload("8^4", (8, 8, 8, 8), "near_identity", 1, 0.3, 0.123,
                    (("composite", 10, 20), ("single", 50), ("single", 10)), 50, 512, 1002, 2002,
                    arnoldi_m=320, ndefinit=200, block=512),
    # HBM-resident lattice: BF16-stored vectors, 200 eigenpairs, 256 noises/level
    "16^3x32": Workload("16^3x32", (16, 16, 16, 32), "near_identity", 2, 0.25, 0.1235,
                        (("composite", 20, 30), ("single", 100), ("single", 16)), 200, 256, 1003, 2003,
                        arnoldi_m=640, ndefinit=420, block=32),
    # near-critical 24^3 x 32: projected composite 50 x 20 (Sec. 4.3), 100 eigenpairs
    "24^3x32": Workload("24^3x32", (24, 24, 24, 32), "near_identity", 3, 0.2, 0.1240,
                        (("deflated_composite", 20, 50), ("single", 100), ("single", 16)), 100, 64, 1004, 2004,
                        arnoldi_m=480, ndefinit=220, block=16),
}


def get(key):
    if key not in WORKLOADS:
        raise KeyError(f"unknown workload {key!r}; choose from {sorted(WORKLOADS)}")
    return WORKLOADS[key]


def gauge(wl):
    return synth.gauge_field(wl.dims, wl.links, wl.gauge_seed, wl.eps)


def setup(h64, wl, log=None):
    """Polynomials [(kind, roots, outer)] and deflation (Zd (k, n) CUDA tensor, lam, pair).

    Order of Sec. 5, step 2: one GMRES run for the single polynomials and
    p_in (2a); PP-Arnoldi eigenpairs with p_in and the Sec. 4 selection (2b);
    p_out from GMRES on A p_in(A), started from the random vector for a plain
    composite, or from a Z4 vector after one Left-right Projection for the
    projected composite (2c).
    """
    S = krylov_setup.Setup(h64)
    v0 = synth.random_unit_vector(wl.n, wl.setup_seed)
    singles = [lv[1] for lv in wl.levels if lv[0] == "single"]
    inners = [lv[1] - 1 for lv in wl.levels if lv[0] != "single"]
    degs = sorted(set(singles + inners))
    roots = dict(zip(degs, S.single_roots(v0, degs)))
    pin = roots[inners[0]] if inners else roots[min(degs)]
    defl = None
    if wl.k > 0:
        Zd, lam, pair = S.eigenpairs(pin, v0, wl.arnoldi_m, wl.ndefinit, kmax=wl.k)
        h64.mpmc_set_deflation_device(Zd, lam, pair)
        # pairs whose left vector cannot be normalised stably (|d_i| small) are dropped
        d = h64.mpmc_deflation_norms()
        keep, pair2 = krylov_setup.Setup.well_conditioned(d, np.asarray(pair))
        if log:
            log(f"setup: {lam.size} of {wl.ndefinit} Ritz pairs accepted (want {wl.k}), "
                f"{keep.size} with |d_i| >= {krylov_setup.DNORM_MIN} (min |d_i| {np.abs(d).min():.3g}); "
                f"|lambda| in [{np.abs(lam).min():.4g}, {np.abs(lam).max():.4g}]")
        if keep.size < lam.size:
            import torch
            Zd = Zd[torch.as_tensor(keep, device=Zd.device)].contiguous()
            lam, pair = lam[keep], pair2
            h64.mpmc_set_deflation_device(Zd, lam, pair)
        defl = (Zd, lam, pair)
    polys = []
    for lv in wl.levels:
        if lv[0] == "single":
            polys.append(("single", roots[lv[1]], None))
            continue
        inner = roots[lv[1] - 1]
        start = v0
        if lv[0] == "deflated_composite":
            if defl is None:
                raise ValueError("a projected composite needs deflation eigenpairs")
            start = S.projected_start(wl.setup_seed)
        outer, _ = S.pp_roots(inner, start, m_out=lv[2])
        polys.append((lv[0], inner, outer))
    return polys, defl


def configure(h, polys, defl, block=None):
    """Load a workload's polynomials and deflation into a handle.

    The roots go in with MPMC_POLY_FP32_COEFS: every handle, whatever its
    precision, then applies the same polynomial (coefficients 1/theta that are
    FP32 numbers), so mixed-precision and FP64 levels estimate the same traces."""
    if defl is not None:
        Z, lam, pair = defl
        if hasattr(Z, "is_cuda") and Z.is_cuda:
            h.mpmc_set_deflation_device(Z, lam, pair)
        else:
            h.mpmc_set_deflation(Z, lam, pair)
    kinds = {"single": G.SINGLE, "composite": G.COMPOSITE, "deflated_composite": G.DEFLATED_COMPOSITE}
    for i, (kind, r, o) in enumerate(polys):
        if kind == "single":
            h.mpmc_set_poly(i, G.SINGLE, r, leja=True, fp32_coefs=True)
        else:
            h.mpmc_set_poly(i, kinds[kind], r, o, leja=True, fp32_coefs=True)
    if block:
        h.mpmc_set_block(block)


# ---------------------------------------------------------------- uneven batch
BATCH_LATTICES = ((4, 4, 4, 4), (6, 6, 6, 6), (8, 8, 8, 8), (8, 8, 8, 16), (12, 12, 12, 12))


def batch_instances(count=64, seed=5, nsamples=32):
    """`count` independent instances for the batched estimate: lattice drawn
    from BATCH_LATTICES, kappa ~ U[0.118, 0.124], eps ~ U[0.2, 0.4], near-identity
    links with their own gauge seed, three levels (composite 20 x 15 = degree
    299, degree 40, degree 8), no deflation, `nsamples` noises per level."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        dims = BATCH_LATTICES[int(rng.integers(len(BATCH_LATTICES)))]
        kappa = float(rng.uniform(0.118, 0.124))
        eps = float(rng.uniform(0.2, 0.4))
        out.append(Workload(f"batch{i}", dims, "near_identity", 100 + i, round(eps, 4), round(kappa, 5),
                            (("composite", 15, 20), ("single", 40), ("single", 8)), 0, nsamples, 5000 + i,
                            6000 + i, block=nsamples))
    return out


def setup_light(h64, wl):
    """Polynomials of a workload without deflation: one GMRES run for the single
    polynomials and p_in, PP-GMRES for p_out (Sec. 5, steps 2a and 2c)."""
    S = krylov_setup.Setup(h64)
    v0 = synth.random_unit_vector(wl.n, wl.setup_seed)
    singles = [lv[1] for lv in wl.levels if lv[0] == "single"]
    inners = [lv[1] - 1 for lv in wl.levels if lv[0] != "single"]
    degs = sorted(set(singles + inners))
    roots = dict(zip(degs, S.single_roots(v0, degs)))
    polys = []
    for lv in wl.levels:
        if lv[0] == "single":
            polys.append(("single", roots[lv[1]], None))
        else:
            inner = roots[lv[1] - 1]
            outer, _ = S.pp_roots(inner, v0, m_out=lv[2])
            polys.append((lv[0], inner, outer))
    return polys
