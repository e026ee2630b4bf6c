"""The probing estimate of Tr p(A) on the GPU (mpmc_trace_probing) against the
oracle's probing_trace on the same probe vectors: FP64 1e-12 relative, FP32
3e-6, BF16-stored 1.5e-2 (the precisions of the polynomial applies), for
single and composite polynomials, colour periods below, at and above the
degree, and ragged last blocks."""

import numpy as np
import pytest

from conftest import links, operator
from oracle import mpmc as M
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import mpmc as G

pytestmark = pytest.mark.gpu

TOL = {G.FP64: 1e-12, G.FP32: 3e-6, G.BF16S: 1.5e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


@pytest.mark.parametrize("prec", [G.FP64, G.FP32, G.BF16S])
@pytest.mark.parametrize("m,block", [(2, 0), (4, 40), (2, 7)])
def test_probing_matches_oracle(prec, m, block):
    dims = (4, 4, 4, 4)
    op = operator(dims, "haar", 2, 0.12)
    single = {"kind": "single", "roots": np.linspace(0.7, 1.4, 4) + 0.1j}
    comp = {"kind": "composite", "inner": np.array([1.1 + 0.1j, 0.8 - 0.05j]), "outer": np.array([0.9, 1.3 + 0.2j])}
    with G.Handle(links(dims, "haar", 2, 0.3), 0.12, prec, 1) as h:
        if block:
            h.mpmc_set_block(block)
        h.mpmc_set_poly(0, G.SINGLE, single["roots"], leja=False)
        h.mpmc_set_poly(1, G.COMPOSITE, comp["inner"], comp["outer"], leja=False)
        got = [h.mpmc_trace_probing(0, m), h.mpmc_trace_probing(1, m)]
    ref = [M.probing_trace(op, single, m), M.probing_trace(op, comp, m)]
    for g, r in zip(got, ref):
        assert abs(g - r) <= TOL[prec] * abs(r), (g, r)


def test_probing_rejects_bad_periods():
    with G.Handle(links((4, 4, 2, 4), "haar", 0, 0.3), 0.12, G.FP64, 1) as h:
        h.mpmc_set_poly(0, G.SINGLE, [1.0, 2.0])
        for m in (0, 3, 4):
            with pytest.raises(G.MpmcError) as e:
                h.mpmc_trace_probing(0, m)
            assert e.value.code == G.MPMC_EINVAL
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_trace_probing(1, 2)
        assert e.value.code == G.MPMC_ESTATE


def test_probing_with_one_colour():
    dims = (4, 2, 2, 4)
    op = operator(dims, "near_identity", 4, 0.12, 0.3)
    single = {"kind": "single", "roots": np.linspace(0.8, 1.2, 3) + 0.05j}
    with G.Handle(links(dims, "near_identity", 4, 0.3), 0.12, G.FP64, 1) as h:
        h.mpmc_set_poly(0, G.SINGLE, single["roots"], leja=False)
        got = h.mpmc_trace_probing(0, 1)
    ref = M.probing_trace(op, single, 1)
    assert abs(got - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("prec", [G.FP64, G.FP32])
def test_distance_colouring_probing_matches_oracle_and_is_exact(prec):
    """Probing with the library's distance-4 colouring: equal to the oracle's
    probing with the same colour table, and (degree 4 <= distance) to the
    exact trace computed densely; a colour table out of range is rejected."""
    from oracle.lattice import dense_A
    dims = (4, 4, 4, 4)
    op = operator(dims, "haar", 2, 0.12)
    colours, nc = G.mpmc_colouring(dims, 4)
    single = {"kind": "single", "roots": np.linspace(0.7, 1.4, 5) + 0.1j}          # degree 4
    comp = {"kind": "composite", "inner": np.array([1.1 + 0.1j, 0.8 - 0.05j]), "outer": np.array([0.9, 1.3 + 0.2j])}
    with G.Handle(links(dims, "haar", 2, 0.3), 0.12, prec, 1) as h:
        h.mpmc_set_block(40)                                      # ragged last block of 12 * nc columns
        h.mpmc_set_poly(0, G.SINGLE, single["roots"], leja=False)
        h.mpmc_set_poly(1, G.COMPOSITE, comp["inner"], comp["outer"], leja=False)
        got = [h.mpmc_trace_probing_colours(0, colours, nc), h.mpmc_trace_probing_colours(1, colours, nc)]
        bad = colours.copy()
        bad[5] = nc
        with pytest.raises(G.MpmcError) as e:
            h.mpmc_trace_probing_colours(0, bad, nc)
        assert e.value.code == G.MPMC_EINVAL
    ref = [M.probing_trace_colours(op, single, colours, nc), M.probing_trace_colours(op, comp, colours, nc)]
    for g, r in zip(got, ref):
        assert abs(g - r) <= TOL[prec] * abs(r), (g, r)
    A = dense_A(links(dims, "haar", 2, 0.3), 0.12)
    P, W = np.zeros_like(A), np.eye(A.shape[0], dtype=np.complex128)
    for th in single["roots"]:
        P += W / th
        W = W - (A @ W) / th
    assert abs(got[0] - np.trace(P)) <= max(TOL[prec], 1e-11) * abs(np.trace(P))
