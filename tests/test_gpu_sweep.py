"""The k_sweep stencil kernels (TMA-staged planes of a 2 x 2 x 2 site block,
site-parallel arithmetic).  The issue-lean kernels are switched off here and
the sweep option set to 8 (k_sweep for every step outside the issue-lean
set), so that every step with a memory input runs
k_sweep / its outer form.

Each case runs the same call with the sweep kernels on and off (the
site-parallel k_step / k_outer) and against the FP64 oracle.  Both kernels
do the same per-site arithmetic in the same hop order, so the stored
vectors agree to FP32 rounding (FMA contraction may differ between the two
kernels): 1e-6 relative.  Level samples differ additionally in the order of
the FP64 per-block dot sums.  Against the oracle the paired bound of
conftest.paired_bound (FP32: bias and noise; BF16-stored: bias, and each
sample within 2e-3 of the summed terms).
"""

import numpy as np
import pytest

from conftest import fp32_resolution, links, operator, paired_bound
from oracle import mpmc as M
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G
from paper_2306_09559_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_ORACLE = {G.FP32: 3e-6, G.BF16S: 1.5e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def _apply_op(dims, bc_t, prec, nrhs, sweep, segment=0, block=0):
    with G.Handle(links(dims, "near_identity", 3, 0.3), 0.124, prec, bc_t) as h:
        if block:
            h.mpmc_set_block(block)
        h.mpmc_set_option(G.OPT_FAST_STENCIL, 0)
        h.mpmc_set_option(G.OPT_SWEEP_STENCIL, 8 * sweep)
        h.mpmc_set_option(G.OPT_SWEEP_SEGMENT, segment)
        X = synth.random_block(12 * int(np.prod(dims)), nrhs, 8)
        Y = h.mpmc_apply_op(X)
        used = h.mpmc_get_option(G.OPT_SWEEP_STENCIL)
        seg = h.mpmc_get_option(G.OPT_SWEEP_SEGMENT)
    return X, Y, used, seg


@pytest.mark.parametrize("dims,bc_t", [((2, 2, 2, 2), -1), ((4, 2, 6, 2), 1), ((4, 4, 4, 8), -1), ((6, 4, 2, 5), 1)])
@pytest.mark.parametrize("prec,nrhs", [(G.FP32, 32), (G.FP32, 40), (G.BF16S, 36), (G.BF16S, 64)])
@pytest.mark.parametrize("segment", [0, 1, 3])
def test_sweep_apply_op(dims, bc_t, prec, nrhs, segment):
    if segment > dims[3]:
        pytest.skip("segment longer than the lattice")
    op = operator(dims, "near_identity", 3, 0.124, 0.3, bc_t)
    X, Y1, used, seg = _apply_op(dims, bc_t, prec, nrhs, 1, segment)
    _, Y0, used0, _ = _apply_op(dims, bc_t, prec, nrhs, 0, segment)
    assert used == 8 and used0 == 0
    assert seg == (segment if segment else seg) and 1 <= seg <= dims[3]
    ref = op(X)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(Y1 - ref)) <= TOL_ORACLE[prec] * scale
    assert np.max(np.abs(Y1 - Y0)) <= 1e-6 * scale


def test_sweep_not_used_where_it_does_not_apply():
    # odd x extent: site-parallel kernel; FP32 odd block width: no 16-byte rows
    _, _, used, _ = _apply_op((3, 2, 2, 4), 1, G.FP32, 8, 1)
    assert used == 0
    _, _, used, _ = _apply_op((4, 4, 2, 4), 1, G.FP32, 7, 1)
    assert used == 0
    _, _, used, _ = _apply_op((4, 4, 2, 4), 1, G.FP64, 8, 1)
    assert used == 0


def test_sweep_segment_range():
    with G.Handle(links((4, 4, 4, 4), "haar", 0, 0.3), 0.12, G.FP32, 1) as h:
        with pytest.raises(G.MpmcError):
            h.mpmc_set_option(G.OPT_SWEEP_STENCIL, 128)
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_set_option(G.OPT_SWEEP_SEGMENT, 5)
        assert e.value.code == G.MPMC_EINVAL
        with pytest.raises(G.MpmcError):
            h.mpmc_set_option(G.OPT_SWEEP_SEGMENT, -1)
        h.mpmc_set_option(G.OPT_SWEEP_SEGMENT, 4)
        assert h.mpmc_get_option(G.OPT_SWEEP_SEGMENT) == 4


def _small_levels():
    from conftest import fp32_polys
    from test_gpu_parity import small_setup
    op, polys, lam, Z, pair = small_setup()
    return op, fp32_polys(polys), lam, Z, pair


@pytest.mark.parametrize("prec", [G.FP32, G.BF16S])
@pytest.mark.parametrize("block,segment", [(32, 0), (16, 1), (64, 3)])
def test_sweep_trace_levels(prec, block, segment):
    """Composite (outer kernel), single levels and deflation through the sweep."""
    from test_gpu_parity import set_polys
    op, polys, lam, Z, pair = _small_levels()
    defl = M.Deflation(op, Z, lam, pair)
    N = 40
    out = {}
    for sweep in (0, 1):
        with G.Handle(links((4, 4, 4, 4), "haar", 0, 0.3), 0.12, prec, 1) as h:
            h.mpmc_set_block(block)
            h.mpmc_set_option(G.OPT_FAST_STENCIL, 0)
            h.mpmc_set_option(G.OPT_SWEEP_STENCIL, 8 * sweep)
            h.mpmc_set_option(G.OPT_SWEEP_SEGMENT, segment)
            h.mpmc_set_deflation(Z, lam, pair)
            set_polys(h, polys)
            out[sweep] = h.mpmc_trace_levels(seed=77, nsamples=N)[2]
            assert h.mpmc_get_option(G.OPT_SWEEP_STENCIL) == 8 * sweep
    for level in range(3):
        ref, hi, lo, dt = M.level_sample_parts(op, polys, level, 77, N, defl)
        mag = np.abs(hi) + np.abs(lo) + np.abs(dt)
        # sweep vs site-parallel: same stored vectors up to FP32 rounding
        rel = 1e-6 if prec == G.FP32 else 1e-2
        assert np.max(np.abs(out[1][level] - out[0][level]) / mag) < rel, level
        if prec == G.FP32:
            paired_bound(out[1][level] - ref, ref, resolution=fp32_resolution(hi, lo))
        else:
            paired_bound(out[1][level] - ref, ref, noise_frac=None)
            assert np.max(np.abs(out[1][level] - ref) / mag) < 2e-3, level


def test_autotune_sets_sweep_options():
    from test_gpu_parity import set_polys
    op, polys, lam, Z, pair = _small_levels()
    with G.Handle(links((4, 4, 4, 4), "haar", 0, 0.3), 0.12, G.FP32, 1) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, polys)
        h.mpmc_set_option(G.OPT_SWEEP_STENCIL, 15)
        cfg = h.mpmc_autotune(64)
        used = h.mpmc_get_option(G.OPT_SWEEP_STENCIL)
        fast = h.mpmc_get_option(G.OPT_FAST_STENCIL)
        seg = h.mpmc_get_option(G.OPT_SWEEP_SEGMENT)
        assert 0 <= used <= 15 and 0 <= fast <= 7 and (used & 7 & ~fast) == 0 and 1 <= seg <= 4
        s = h.mpmc_trace_levels(seed=5, nsamples=20)[2]
    ref = M.level_samples(op, polys, 2, 5, 20)
    assert np.max(np.abs(s[2] - ref)) < 1e-5 * op.n
    assert cfg["nb"] in (16, 32, 64)
