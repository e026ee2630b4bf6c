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
