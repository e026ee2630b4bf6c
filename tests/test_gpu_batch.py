"""Batches of independent instances (mpmc_batch_*): the multilevel traces of
handles with different lattices, kappas, polynomials, deflation and
precision run as parallel branches of one captured CUDA graph.  Each
handle's means and variances must equal what mpmc_trace_levels returns for
it alone (same kernels, same launch shapes, same summation order: 1e-13 of
the level's size), on the capturing call, on a replay, and after a change
to one handle (which recaptures the graph)."""

import numpy as np
import pytest

from conftest import links
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def _instances():
    from test_gpu_parity import set_polys, small_setup
    op, polys, lam, Z, pair = small_setup()
    hs = []
    h = G.Handle(links((4, 4, 4, 4), "haar", 0, 0.3), 0.12, G.FP32, 1)
    h.mpmc_set_deflation(Z, lam, pair)
    set_polys(h, polys)
    h.mpmc_set_block(16)
    hs.append(h)
    h = G.Handle(links((2, 4, 2, 4), "near_identity", 5, 0.3), 0.121, G.FP64, -1)
    h.mpmc_set_poly(0, G.SINGLE, np.linspace(0.6, 1.4, 9) + 0.05j)
    h.mpmc_set_poly(1, G.SINGLE, np.linspace(0.7, 1.3, 4) + 0.02j)
    hs.append(h)
    h = G.Handle(links((6, 4, 4, 2), "near_identity", 6, 0.25), 0.119, G.BF16S, 1)
    h.mpmc_set_poly(0, G.COMPOSITE, np.linspace(0.6, 1.4, 3) + 0.1j, np.linspace(0.5, 1.5, 4))
    h.mpmc_set_poly(1, G.SINGLE, np.linspace(0.6, 1.4, 5) + 0.1j)
    h.mpmc_set_poly(2, G.SINGLE, np.linspace(0.8, 1.2, 2) + 0.1j)
    h.mpmc_set_block(32)
    hs.append(h)
    return hs


def _alone(hs, seed, N, first):
    out = []
    for h in hs:
        m, v, _ = h.mpmc_trace_levels(seed, N, first, want_samples=False)
        out.append((m, v))
    return out


def _compare(mean, var, ref):
    for i, (m, v) in enumerate(ref):
        L = m.size
        scale = np.maximum(np.abs(m), 1.0)
        assert np.all(np.abs(mean[i, :L] - m) <= 1e-13 * scale), i
        assert np.allclose(var[i, :L], v, rtol=1e-12, atol=0, equal_nan=True), i


def test_batch_matches_each_handle_alone():
    hs = _instances()
    try:
        ref = _alone(hs, 41, 40, 3)
        with G.Batch(hs) as b:
            m1, v1 = b.mpmc_batch_trace_levels(41, 40, 3)     # plain run, capture, replay
            n1 = b.mpmc_batch_launch_count()
            m2, v2 = b.mpmc_batch_trace_levels(41, 40, 3)     # replay of the same graph
            n2 = b.mpmc_batch_launch_count()
            assert n1 > 0 and n2 == 2 * n1
            _compare(m1, v1, ref)
            _compare(m2, v2, ref)
            # a new noise block and a changed handle: the graph is captured again
            hs[1].mpmc_set_poly(1, G.SINGLE, np.linspace(0.7, 1.3, 6) + 0.02j)
            ref3 = _alone(hs, 42, 24, 0)
            m3, v3 = b.mpmc_batch_trace_levels(42, 24, 0)
            _compare(m3, v3, ref3)
    finally:
        for h in hs:
            h.close()


def test_batch_recaptures_after_plain_calls_reallocate_buffers():
    """Plain calls on a batched handle (a longer trace, an apply with a narrower
    block, deflation dots) free and reallocate buffers the captured graph was
    recorded with; the next identical batch call must recapture, not replay
    kernels on the old addresses."""
    hs = _instances()
    rng = np.random.default_rng(3)
    try:
        ref = _alone(hs, 41, 40, 3)
        with G.Batch(hs) as b:
            m1, v1 = b.mpmc_batch_trace_levels(41, 40, 3)
            _compare(m1, v1, ref)
            hs[0].mpmc_trace_levels(9, 300, 0, want_samples=False)          # longer sample buffer
            for h in (hs[0], hs[2]):                                         # narrower work block
                B = rng.standard_normal((h.n, 3)) + 1j * rng.standard_normal((h.n, 3))
                h.mpmc_apply_poly(1, B)
            hs[0].mpmc_deflation_dots(5, 1, 0, 7, hs[0].k)                  # other deflation width
            m2, v2 = b.mpmc_batch_trace_levels(41, 40, 3)
            _compare(m2, v2, ref)
            m3, v3 = b.mpmc_batch_trace_levels(41, 40, 3)                   # replay of the new graph
            _compare(m3, v3, ref)
    finally:
        for h in hs:
            h.close()


@pytest.mark.parametrize("prec", [G.FP64, G.FP32])
def test_batch_instances_match_the_oracle(prec):
    """One instance of each cheap lattice class of the 64-instance batch (4^4 and
    6^4: near-identity links, its own kappa, composite 15 x 20, degrees 40 and 8,
    32 noises), with roots from the oracle's setup, run as a batch: each level's
    mean equals the oracle's mean over the same noise, to 1e-12 of the summed
    terms in FP64, and within the paired bias bound in FP32 (the differences of
    the per-sample values of the same handle traced alone, which the batch
    reproduces bit for bit, against the oracle's samples)."""
    from conftest import fp32_resolution, paired_bound
    from oracle import krylov as K
    from oracle import mpmc as M
    from oracle.lattice import WilsonOperator
    from paper_2306_09559_gb300 import synth, workloads
    from test_gpu_parity import set_polys
    insts = workloads.batch_instances()
    pick = [next(w for w in insts if w.dims == d) for d in ((4, 4, 4, 4), (6, 6, 6, 6))]
    N, seed = 32, 7
    hs, oracle = [], []
    try:
        for w in pick:
            U = workloads.gauge(w)
            op = WilsonOperator(U, w.kappa)
            b0 = synth.random_unit_vector(op.n, w.setup_seed)
            p40, p8, p_in = K.gmres_polynomials(op, b0, [40, 8, 14])
            p_out, _, _ = K.pp_gmres_roots(op, p_in, b0, m_out=20)
            polys = [{"kind": "composite", "inner": p_in, "outer": p_out},
                     {"kind": "single", "roots": p40}, {"kind": "single", "roots": p8}]
            if prec != G.FP64:
                from conftest import fp32_polys
                polys = fp32_polys(polys)
            h = G.Handle(U, w.kappa, prec)
            set_polys(h, polys)
            h.mpmc_set_block(N)
            hs.append(h)
            oracle.append([M.level_sample_parts(op, polys, l, seed, N) for l in range(3)])
        alone = [h.mpmc_trace_levels(seed, N, 0)[2] for h in hs]
        with G.Batch(hs) as b:
            mean, _ = b.mpmc_batch_trace_levels(seed, N, 0)
        for i in range(len(hs)):
            for l in range(3):
                ref, hi, lo, _ = oracle[i][l]
                mag = np.mean(np.abs(hi) + np.abs(lo))
                if prec == G.FP64:
                    assert abs(mean[i, l] - ref.mean()) <= 1e-12 * mag, (i, l)
                else:
                    assert abs(mean[i, l] - alone[i][l].mean()) <= 1e-13 * mag, (i, l)
                    paired_bound(alone[i][l] - ref, ref, resolution=fp32_resolution(hi, lo))
    finally:
        for h in hs:
            h.close()


def test_batch_rejects_bad_arguments():
    import ctypes
    L = G.lib()
    b = ctypes.c_void_p()
    assert L.mpmc_batch_create(ctypes.byref(b), 0, None) == G.MPMC_EINVAL
    assert L.mpmc_batch_trace_levels(None, 1, 4, 0, None, None) == G.MPMC_EINVAL
    assert L.mpmc_batch_destroy(None) == G.MPMC_EINVAL


def test_batch_rejects_a_handle_on_the_legacy_default_stream():
    import ctypes
    h = G.Handle(links((4, 4, 2, 4), "haar", 0, 0.3), 0.12, G.FP32, 1)
    try:
        h.mpmc_set_stream(1)        # cudaStreamLegacy: usable alone, but it cannot be captured
        L = G.lib()
        arr = (ctypes.c_void_p * 1)(h._h)
        b = ctypes.c_void_p()
        assert L.mpmc_batch_create(ctypes.byref(b), 1, ctypes.cast(arr, ctypes.c_void_p)) == G.MPMC_EINVAL
    finally:
        h.close()
