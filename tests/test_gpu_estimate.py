"""The sequential multilevel estimate on the library (mpmc_trace_level, Sec. 5
step 3): each level's estimate equals the oracle's mean over the same noise
indices plus its exact correction (1e-12 relative to the summed terms, the
FP64 per-sample bound), and the total standard error meets the tolerance."""

import numpy as np
import pytest

from oracle import mpmc as M
from paper_2306_09559_gb300 import build
from paper_2306_09559_gb300 import estimate as E
from paper_2306_09559_gb300 import mpmc as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    G.lib()


def test_trace_level_matches_trace_levels():
    from test_gpu_parity import handle, set_polys, small_setup
    op, polys, lam, Z, pair = small_setup()
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, polys)
        mean, var, s = h.mpmc_trace_levels(8, 21, 2)
        for level in range(3):
            m1, v1, s1 = h.mpmc_trace_level(level, 8, 21, 2)
            assert np.max(np.abs(s1 - s[level])) < 1e-12 * op.n
            assert abs(m1 - mean[level]) < 1e-12 * op.n and np.isclose(v1, var[level], rtol=1e-12)


def test_sequential_estimate_on_the_gpu_matches_the_oracle():
    from test_gpu_parity import handle, set_polys, small_setup
    op, polys, lam, Z, pair = small_setup()
    defl = M.Deflation(op, Z, lam, pair)
    with handle((4, 4, 4, 4)) as h:
        h.mpmc_set_deflation(Z, lam, pair)
        set_polys(h, polys)
        _, var, _ = h.mpmc_trace_levels(3, 16, 1000)
        eps = float(np.sqrt(np.sum(var) / 30.0))
        res = E.sequential_estimate(E.library_sampler(h, 3), [0, 1, 2], eps, chunk=24)
    assert res["err"] <= eps * (1 + 1e-12)
    for lv in res["levels"]:
        ref, hi, lo, dt = M.level_sample_parts(op, polys, lv["level"], 3, lv["n"], defl)
        est = np.mean(ref) + M.exact_correction(polys, lv["level"], defl)
        scale = np.mean(np.abs(hi) + np.abs(lo) + np.abs(dt))
        assert abs(lv["estimate"] - est) < 1e-12 * scale, lv


def test_choose_degree_minimises_the_eq3_cost():
    """The degree of p_2 picked from the Eq. (3) cost of pilot runs is the one
    that minimises that cost computed by the oracle (its own samples of the same
    noise, its own multilevel_cost), and the library's costs agree with the
    oracle's to 1e-8."""
    from conftest import operator
    from oracle import krylov as K
    from paper_2306_09559_gb300 import synth
    from test_gpu_parity import handle, set_polys
    op = operator((4, 4, 4, 4), "haar", 0, 0.12)
    b0 = synth.random_unit_vector(op.n, 17)
    cands = [3, 6, 12, 20, 30]
    roots = dict(zip(cands + [2], K.gmres_polynomials(op, b0, cands + [2])))
    p_in = K.gmres_polynomials(op, b0, [5])[0]
    p_out = K.pp_gmres_roots(op, p_in, b0, m_out=8)[0]
    eps, seed, pilot = 1.0, 404, 40
    costs_o = {}
    for d in cands:
        polys = [{"kind": "composite", "inner": p_in, "outer": p_out},
                 {"kind": "single", "roots": roots[d]}, {"kind": "single", "roots": roots[2]}]
        var = [np.var(M.level_samples(op, polys, l, seed, pilot).real, ddof=1) for l in range(3)]
        C = [M.spec_matvecs(polys[l]) + (M.spec_matvecs(polys[l + 1]) if l < 2 else 0) for l in range(3)]
        costs_o[d] = M.multilevel_cost(var, C, eps)
    with handle((4, 4, 4, 4)) as h:
        set_polys(h, [{"kind": "composite", "inner": p_in, "outer": p_out},
                      {"kind": "single", "roots": roots[cands[0]]}, {"kind": "single", "roots": roots[2]}])
        best, costs = E.choose_degree(h, 1, cands, lambda d: roots[d], eps, seed, pilot=pilot)
    assert best == min(costs_o, key=costs_o.get)
    for d in cands:
        assert abs(costs[d] - costs_o[d]) <= 1e-8 * costs_o[d], d
