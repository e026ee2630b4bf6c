"""Failure detection of the bounded device waits (no GPU fault involved).

The t-sweep stencil kernels wait on an mbarrier for every TMA plane copy,
with a bound.  A test hook (MPMC_OPT_TEST_SKIP_COPY) makes each CTA's
producer leave out one plane copy, so the consumers' wait for it runs out
with no copy in flight into that buffer; with a short wait limit the call
returns MPMC_ETIMEOUT quickly.  The CTA waits (bounded) for the copies it
did issue before it leaves, so the context stays usable: the next call on
the same handle, hook off, gives exactly the samples of a fresh handle and
matches the oracle within the paired bound."""

import numpy as np
import pytest

from conftest import fp32_polys, fp32_resolution, links, paired_bound
from oracle import mpmc as M
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def _handle(prec, Z, lam, pair, polys, block=16):
    from test_gpu_parity import set_polys
    h = G.Handle(links((4, 4, 4, 4), "haar", 0, 0.3), 0.12, prec, 1)
    h.mpmc_set_block(block)
    h.mpmc_set_option(G.OPT_FAST_STENCIL, 7)
    h.mpmc_set_option(G.OPT_SWEEP_STENCIL, 7)
    h.mpmc_set_option(G.OPT_SWEEP_SEGMENT, 4)           # planes 0 .. 5 in each CTA's ring
    h.mpmc_set_deflation(Z, lam, pair)
    set_polys(h, polys)
    return h


@pytest.mark.parametrize("skip", [1, 2, 5])
@pytest.mark.parametrize("sweep", [7, 23, 39, 71])
def test_a_wait_that_runs_out_returns_etimeout_and_the_handle_recovers(skip, sweep):
    """Every t-sweep form (links from global memory, staged, warp-per-site with blocks of 32,
    two sites per warp)."""
    from test_gpu_parity import small_setup
    op, polys, lam, Z, pair = small_setup()
    polys = fp32_polys(polys)
    block = 32 if sweep & 32 else 16
    N = block + block // 2            # two blocks of `block` columns, the second one ragged
    with _handle(G.FP32, Z, lam, pair, polys, block) as h, _handle(G.FP32, Z, lam, pair, polys, block) as fresh:
        for hh in (h, fresh):
            hh.mpmc_set_option(G.OPT_SWEEP_STENCIL, sweep)
        assert h.mpmc_get_option(G.OPT_SWEEP_STENCIL) == sweep
        h.mpmc_set_option(G.OPT_WAIT_LIMIT, 20000)          # 2e7 cycles: about 10 ms
        assert h.mpmc_get_option(G.OPT_WAIT_LIMIT) == 20000
        h.mpmc_set_option(G.OPT_TEST_SKIP_COPY, skip)
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_trace_levels(seed=3, nsamples=N)
        assert e.value.code == G.MPMC_ETIMEOUT
        h.mpmc_set_option(G.OPT_TEST_SKIP_COPY, 0)
        got = h.mpmc_trace_levels(seed=3, nsamples=N)[2]
        ref_gpu = fresh.mpmc_trace_levels(seed=3, nsamples=N)[2]
    assert np.array_equal(got, ref_gpu)
    defl = M.Deflation(op, Z, lam, pair)
    for level in range(3):
        ref, hi, lo, _ = M.level_sample_parts(op, polys, level, 3, N, defl)
        paired_bound(got[level] - ref, ref, resolution=fp32_resolution(hi, lo))


def test_wait_options_are_checked():
    with G.Handle(links((4, 4, 2, 4), "haar", 0, 0.3), 0.12, G.FP32, 1) as h:
        for bad in (0, 4000001):
            with pytest.raises(G.MpmcError) as e:
                h.mpmc_set_option(G.OPT_WAIT_LIMIT, bad)
            assert e.value.code == G.MPMC_EINVAL
        with pytest.raises(G.MpmcError):
            h.mpmc_set_option(G.OPT_TEST_SKIP_COPY, -1)
        assert h.mpmc_get_option(G.OPT_WAIT_LIMIT) == 4000000
        assert h.mpmc_get_option(G.OPT_TEST_SKIP_COPY) == 0
