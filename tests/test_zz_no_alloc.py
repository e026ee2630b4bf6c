"""The allocation-free entry point agrees with mpmc_trace_levels.

mpmc_trace_poly_noalloc serves callers that cannot call cudaMalloc (a
framework owns the device memory, or cudaMalloc's implicit synchronisation
is not acceptable on their path): it keeps its scratch in a fixed device
array instead of allocating.  Two calls in a row must both reproduce the
samples of the existing entry point for the same polynomial and noise, to
the tolerance of the FP64 parity tests (1e-12 of the size n of the summed
terms), whatever the previous call left in the array.
"""

import numpy as np
import pytest

from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G
from paper_2306_09559_gb300 import synth

pytestmark = pytest.mark.gpu


def _roots():
    from oracle import krylov as K
    from oracle.lattice import WilsonOperator
    U = synth.gauge_field((4, 4, 4, 4), "haar", seed=3)
    op = WilsonOperator(U, 0.12)
    return U, K.gmres_polynomials(op, synth.random_unit_vector(op.n, 5), [17])[0]


def test_noalloc_matches_trace_levels_two_calls():
    torch = pytest.importorskip("torch")
    build.build()
    U, roots = _roots()
    n = 12 * 256
    with G.Handle(U, 0.12, G.FP64) as h:
        h.mpmc_set_poly(0, G.SINGLE, roots, leja=False)
        ref_a = h.mpmc_trace_levels(seed=77, nsamples=70, first=3)[2][0]
        ref_b = h.mpmc_trace_levels(seed=77, nsamples=9, first=100)[2][0]
    # call 1: host links and host result
    got_a = G.mpmc_trace_poly_noalloc(U, 0.12, roots, seed=77, level=0, first=3, nsamples=70)
    # call 2: device links and device result, right after (the array holds call 1's data)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    out = torch.zeros(9, dtype=torch.complex128, device="cuda")
    G.mpmc_trace_poly_noalloc(Ud, 0.12, roots, seed=77, level=0, first=100, nsamples=9, out=out)
    torch.cuda.synchronize()
    got_b = out.cpu().numpy()
    assert np.max(np.abs(got_a - ref_a)) < 1e-12 * n
    assert np.max(np.abs(got_b - ref_b)) < 1e-12 * n


def test_noalloc_rejects_a_lattice_beyond_the_array():
    import ctypes
    build.build()
    L = G.lib()
    # 32^4: two chain vectors alone need 2 * 12 * 2^20 * 16 B = 384 MiB > 32 MiB; the size
    # check comes before any copy, so a one-entry dummy buffer stands in for the links
    dims = (ctypes.c_int * 4)(32, 32, 32, 32)
    dummy = np.zeros(1, dtype=np.complex128)
    roots = np.array([1.0 + 0j, 2.0 + 0j])
    out = np.zeros(1, dtype=np.complex128)
    rc = L.mpmc_trace_poly_noalloc(dims, G._ptr(dummy), 0.12, 1, G._ptr(roots), 2, ctypes.c_uint64(1), 0, 0, 1,
                                   G._ptr(out), 0, None)
    assert rc == G.MPMC_EINVAL
