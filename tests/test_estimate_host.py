"""Host logic of the sequential multilevel estimate (Sec. 5, step 3) and of
the sample allocation (Eq. (3)), with a deterministic synthetic sampler whose
samples depend only on (level, index) like the library's."""

import math

import numpy as np

from oracle import mpmc as M
from paper_2306_09559_gb300 import estimate as E

SIG = [4.0, 1.5, 0.3]


def sampler(level, first, count):
    out = np.empty(count, dtype=np.complex128)
    for i in range(count):
        r = np.random.Generator(np.random.PCG64([level, first + i]))
        out[i] = 10.0 * level + SIG[level] * r.normal() + 1j * r.normal()
    return out, 0.5j


def test_stop_point_is_the_first_check_point_meeting_the_tolerance():
    s, _ = sampler(0, 0, 400)
    for tol in (0.9, 0.5, 0.3):
        n = E.stop_point(s.real, tol, 3, 3)
        assert n is not None and (n - 3) % 3 == 0
        assert E.standard_error(s.real, n) <= tol
        assert all(E.standard_error(s.real, m) > tol for m in range(3, n, 3))


def test_sequential_estimate_meets_the_tolerance_and_the_split():
    eps = 0.2
    res = E.sequential_estimate(sampler, [0, 1, 2], eps, chunk=16)
    assert res["err"] <= eps + 1e-12
    cur = 0.0
    for k, lv in enumerate(res["levels"]):
        tol = math.sqrt((eps * eps - cur) / (3 - k))
        assert abs(lv["tol"] - tol) < 1e-12
        start, step = E.schedule(k)
        assert lv["n"] >= start and (lv["n"] - start) % step == 0
        s, c = sampler(lv["level"], 0, lv["n"])
        assert lv["estimate"] == np.mean(s) + c
        assert lv["se"] <= tol
        cur += lv["se"] ** 2
    # chunk size does not change where the rule stops
    res2 = E.sequential_estimate(sampler, [0, 1, 2], eps, chunk=5)
    assert [x["n"] for x in res2["levels"]] == [x["n"] for x in res["levels"]]


def test_allocation_reaches_the_multilevel_cost():
    v, c, eps = [0.8, 3.0, 20.0], [500.0, 60.0, 10.0], 0.05
    n, cost = E.allocation(v, c, eps)
    assert abs(cost - M.multilevel_cost(v, c, eps)) < 1e-9 * cost
    # with N_l samples the total variance sum V_l / N_l is at most eps^2
    assert np.sum(np.array(v) / n) <= eps ** 2 * (1 + 1e-12)


def test_precision_corrected_level_is_the_fp64_mean_for_paired_samples():
    """With fake handles: mixed samples m, FP64 samples f on the same noise; the
    corrected estimate is mean(m) + mean(f - m)[:n], its variance the three-term
    formula, and with n = N it equals the FP64 mean exactly."""
    import numpy as np
    from paper_2306_09559_gb300 import estimate as E

    rng = np.random.default_rng(1)
    f = rng.standard_normal(40) * 2.0 + 5.0
    m = f + 0.03 + 1e-3 * rng.standard_normal(40)          # a biased mixed path

    class Fake:
        def __init__(self, s, corr):
            self.s, self.corr = s, corr

        def mpmc_trace_level(self, level, seed, n, first):
            x = self.s[first:first + n].astype(complex)
            return np.mean(x) + self.corr, np.var(x.real, ddof=1), x

    r = E.precision_corrected_level(Fake(m, 0.5), Fake(f, 0.5), 0, 7, 40, 40)
    assert abs(r["estimate"] - (np.mean(f) + 0.5)) < 1e-12
    r = E.precision_corrected_level(Fake(m, 0.5), Fake(f, 0.5), 0, 7, 40, 5)
    d = f[:5] - m[:5]
    assert abs(r["estimate"] - (np.mean(m) + 0.5 + np.mean(d))) < 1e-12
    v = np.var(m, ddof=1) / 40 + np.var(d, ddof=1) / 5 + 2 * np.cov(m[:5], d)[0, 1] / 40
    assert abs(r["se"] ** 2 - v) < 1e-12
    assert E.correction_samples(4.0, 1e-6, 1.0, 20.0, 64) == 2
    assert E.correction_samples(4.0, 4.0, 1.0, 1.0, 64) == 64
