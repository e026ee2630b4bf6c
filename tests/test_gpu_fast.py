"""The issue-lean stencil kernels (packed FP32x2 arithmetic, compile-time
block width, per-block Z4 word table) and their t-sweep form.

They run the trace-mode steps (the noise-started first step, the dotted
steps of a single chain, the inner steps and the outer step of a composite
chain).  Each case runs the same trace with the kernels on and off (the
site-parallel k_step / k_outer) and against the FP64 oracle.  Per-component
rounding is that of scalar FMAs but the hopping sums are grouped
differently, so the two agree to FP32 rounding of the summed terms:
|s_on - s_off| <= 2e-6 (|b^H p_l b| + |b^H p_{l+1} b| + |deflation term|)
per sample for FP32 storage, 2e-3 for BF16 storage (the stored vectors
round to bf16 at every step, stochastically).  Against the oracle: the
paired bound of conftest.paired_bound (bias, and noise within the FP32
resolution of a sample) for FP32 storage; for BF16 storage its bias part,
and each sample within 2e-3 of the summed terms.
"""

import numpy as np
import pytest

from conftest import fp32_polys, fp32_resolution, links, operator, paired_bound
from oracle import krylov as K
from oracle import mpmc as M
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G
from paper_2306_09559_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def _setup(dims, bc_t):
    """Oracle roots (with FP32 product-form coefficients, the polynomial every handle of these
    tests applies) and selected deflation pairs (Sec. 4) on Haar links, kappa 0.12."""
    from test_gpu_parity import small_setup
    if dims == (4, 4, 4, 4) and bc_t == 1:
        op, polys, lam, Z, pair = small_setup()
        return op, fp32_polys(polys), lam, Z, pair
    op = operator(dims, "haar", 0, 0.12, 0.3, bc_t)
    b0 = synth.random_unit_vector(op.n, 17)
    p_hi, p_lo, p_in = K.gmres_polynomials(op, b0, [14, 6, 3])
    p_out, _, _ = K.pp_gmres_roots(op, p_in, b0, m_out=4)
    lam, Z = K.pp_arnoldi_ritz(op, p_in, b0, m=60, nev=8)
    lam_s, Z_s, pair = K.select_deflation(op, op.gamma5, lam, Z)
    polys = [{"kind": "composite", "inner": p_in, "outer": p_out},
             {"kind": "single", "roots": p_hi},
             {"kind": "single", "roots": p_lo}]
    return op, fp32_polys(polys), lam_s, Z_s, pair


def _deflation(setup):
    op, _, lam, Z, pair = setup
    return M.Deflation(op, Z, lam, pair) if lam.size else None


def _trace(dims, bc_t, prec, block, fast, sl=1, N=None, setup=None, defl=True, sweep=0, segment=0):
    from test_gpu_parity import set_polys
    op, polys, lam, Z, pair = setup
    with G.Handle(links(dims, "haar", 0, 0.3), 0.12, prec, bc_t) as h:
        h.mpmc_set_block(block)
        h.mpmc_set_option(G.OPT_FAST_STENCIL, fast)
        h.mpmc_set_option(G.OPT_FAST_SITES, sl)
        h.mpmc_set_option(G.OPT_SWEEP_STENCIL, sweep)
        h.mpmc_set_option(G.OPT_SWEEP_SEGMENT, segment)
        if defl and lam.size:
            h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, polys)
        s = h.mpmc_trace_levels(seed=31, nsamples=N or block)[2]
        used = (h.mpmc_get_option(G.OPT_FAST_STENCIL), h.mpmc_get_option(G.OPT_SWEEP_STENCIL),
                h.mpmc_get_option(G.OPT_SWEEP_SEGMENT))
    return s, used


def _check(setup, got, ref_gpu, prec, N, rel):
    op, polys = setup[0], setup[1]
    defl = _deflation(setup)
    for level in range(3):
        ref, hi, lo, dt = M.level_sample_parts(op, polys, level, 31, N, defl)
        mag = np.abs(hi) + np.abs(lo) + np.abs(dt)
        assert np.max(np.abs(got[level] - ref_gpu[level]) / mag) < rel, level
        if prec == G.FP32:
            paired_bound(got[level] - ref, ref, resolution=fp32_resolution(hi, lo))
        else:
            paired_bound(got[level] - ref, ref, noise_frac=None)
            assert np.max(np.abs(got[level] - ref) / mag) < 2e-3, level


CASES = [((4, 4, 4, 4), 1, 16), ((4, 4, 4, 4), 1, 32), ((3, 5, 2, 3), -1, 16), ((2, 2, 2, 2), -1, 32),
         ((6, 4, 2, 2), 1, 64)]


@pytest.mark.parametrize("dims,bc_t,block", CASES)
@pytest.mark.parametrize("prec", [G.FP32, G.BF16S])
@pytest.mark.parametrize("sl", [1, 2, 4])
def test_fast_matches_site_parallel_and_oracle(dims, bc_t, block, prec, sl):
    setup = _setup(dims, bc_t)
    N = block + block // 2          # two blocks, the second one ragged
    on, used = _trace(dims, bc_t, prec, block, 7, sl, N, setup=setup)
    off, used0 = _trace(dims, bc_t, prec, block, 0, sl, N, setup=setup)
    assert used[0] == 7 and used0[0] == 0
    _check(setup, on, off, prec, N, 2e-6 if prec == G.FP32 else 2e-3)


@pytest.mark.parametrize("dims,bc_t,block", [((4, 4, 4, 4), 1, 16), ((4, 4, 4, 4), 1, 32), ((2, 2, 2, 2), -1, 32),
                                             ((6, 4, 2, 5), -1, 16), ((4, 2, 6, 2), 1, 64)])
@pytest.mark.parametrize("prec", [G.FP32, G.BF16S])
@pytest.mark.parametrize("segment", [0, 1, 3])
@pytest.mark.parametrize("sweep", [7, 23, 39, 71])
def test_fast_sweep_matches_fast_and_oracle(dims, bc_t, block, prec, segment, sweep):
    """The t-sweep form (TMA-staged planes; sweep 23 also stages each plane's
    links in shared memory, sweep 39 runs the warp-per-site form of that at
    blocks of 32 or more and the sweep-23 form below, sweep 71 the
    two-sites-per-warp form) against k_fast and the oracle: same arithmetic per site up to the order of the hop sum and of the
    FP64 dot sums."""
    if segment > dims[3]:
        pytest.skip("segment longer than the lattice")
    setup = _setup(dims, bc_t)
    N = block + block // 2
    sw, used = _trace(dims, bc_t, prec, block, 7, 1, N, setup=setup, sweep=sweep, segment=segment)
    plain, used0 = _trace(dims, bc_t, prec, block, 7, 1, N, setup=setup, sweep=0)
    assert used[:2] == (7, 23 if sweep == 39 and block < 32 else sweep) and used0[:2] == (7, 0)
    assert 1 <= used[2] <= dims[3] and (segment == 0 or used[2] == segment)
    _check(setup, sw, plain, prec, N, 2e-6 if prec == G.FP32 else 2e-3)


@pytest.mark.parametrize("block", [128, 256, 512, 1024])
@pytest.mark.parametrize("mask", [0, 7, 23, 39, 71])
def test_fast_wide_blocks(block, mask):
    """The block widths the 8^4 benchmark runs (512, 1024) and the ones between:
    issue-lean kernels (plain and t-sweep) against the site-parallel ones, and
    each against the oracle on the same noise (paired bound)."""
    dims = (4, 4, 2, 4)
    setup = _setup(dims, 1)
    # none, t-sweep, t-sweep with links in shared memory, its warp-per-site and two-sites-per-warp forms
    on, used = _trace(dims, 1, G.FP32, block, 7, 1, block, setup=setup, defl=False, sweep=mask)
    off, _ = _trace(dims, 1, G.FP32, block, 0, 1, block, setup=setup, defl=False)
    assert used[:2] == (7, mask)
    n = 12 * int(np.prod(dims))
    op, polys = setup[0], setup[1]
    for level in range(3):
        scale = n + np.max(np.abs(off[level]))
        assert np.max(np.abs(on[level] - off[level])) < 1e-5 * scale, level
        ref, hi, lo, _ = M.level_sample_parts(op, polys, level, 31, block)
        paired_bound(on[level] - ref, ref, resolution=fp32_resolution(hi, lo))
        paired_bound(off[level] - ref, ref, resolution=fp32_resolution(hi, lo))


def test_fast_not_used_where_it_does_not_apply():
    setup = _setup((4, 4, 4, 4), 1)
    _, used = _trace((4, 4, 4, 4), 1, G.FP32, 24, 7, 1, 24, setup=setup)
    assert used[0] == 0                  # block width outside the compiled set
    _, used = _trace((4, 4, 4, 4), 1, G.FP64, 32, 7, 1, 32, setup=setup)
    assert used[0] == 0                  # FP64 keeps the site-parallel kernel


@pytest.mark.parametrize("mask", [1, 2, 4, 5])
def test_fast_per_class_masks(mask):
    """Any subset of step classes (dotted, undotted inner, outer) on the issue-lean
    kernels, the rest on the site-parallel ones, gives the same samples."""
    dims = (4, 4, 4, 4)
    setup = _setup(dims, 1)
    N = 48
    part, used = _trace(dims, 1, G.FP32, 32, mask, 1, N, setup=setup, sweep=mask)
    off, _ = _trace(dims, 1, G.FP32, 32, 0, 1, N, setup=setup)
    assert used[:2] == (mask, mask)
    _check(setup, part, off, G.FP32, N, 2e-6)


def test_fast_sites_option_range():
    with G.Handle(links((4, 4, 4, 4), "haar", 0, 0.3), 0.12, G.FP32, 1) as h:
        for bad in (-1, 8):
            with pytest.raises(G.MpmcError):
                h.mpmc_set_option(G.OPT_FAST_STENCIL, bad)
        for bad in (0, 17):
            with pytest.raises(G.MpmcError) as e:
                h.mpmc_set_option(G.OPT_FAST_SITES, bad)
            assert e.value.code == G.MPMC_EINVAL
        h.mpmc_set_option(G.OPT_FAST_SITES, 3)
        assert h.mpmc_get_option(G.OPT_FAST_SITES) == 3
